// C ABI of libnegf: context, batch layout, and the drivers of the open boundary
// conditions, the RGF sweeps (Eqs. (1)-(2) of the paper) and the observables.
// Every arithmetic step runs in the kernels of this library; the host only
// validates arguments, lays out the packed batch (integer prefix sums) and
// sequences launches on the caller's stream.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "negf_internal.cuh"

using namespace negf;

namespace {

// ---------------------------------------------------------------------------
// error plumbing
// ---------------------------------------------------------------------------
thread_local std::string g_tls_error;

negf_status fail(Ctx* c, negf_status code, const std::string& msg) {
  if (c) c->last_error = msg;
  g_tls_error = msg;
  return code;
}

// launch check that also counts the kernel for the context's launch counter
#define KCHECK() do { ++ctx->launches; CU(cudaGetLastError()); } while (0)

#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return fail(ctx, NEGF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ---------------------------------------------------------------------------
// one device of the (possibly uneven) batch, as the kernels see it
// ---------------------------------------------------------------------------
struct DevView {
  const zc* Hd;   // block 0 of this device
  const zc* Hu;
  const zc* Sd;   // NULL => identity
  const zc* Su;   // NULL => zero
  const double* E;
  double eta;
  int nb, b;
};

struct ScatView {
  const zc* sigR;        // NULL or this device's block 0 (energy 0)
  const zc* sigL;
  const double* scale;   // NULL or [ne][nb] of this device
  long long e_stride;    // elements between energies (0 = shared)
};

struct Layout {
  int ndev;
  std::vector<long long> off;   // 8*(ndev+1)
};

negf_status make_layout(Ctx* ctx, const negf_system* sys, Layout& L) {
  if (!sys) return fail(ctx, NEGF_ERR_ARG, "negf_system is NULL");
  if (sys->ndev < 1) return fail(ctx, NEGF_ERR_ARG, "ndev must be >= 1");
  if (!sys->nb || !sys->bs || !sys->ne) return fail(ctx, NEGF_ERR_ARG, "nb/bs/ne host arrays are NULL");
  L.ndev = sys->ndev;
  L.off.assign(8 * (size_t)(sys->ndev + 1), 0);
  long long acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int d = 0; d < sys->ndev; ++d) {
    const long long nb = sys->nb[d], b = sys->bs[d], ne = sys->ne[d];
    if (nb < 1 || b < 1 || b > 512 || ne < 0)
      return fail(ctx, NEGF_ERR_ARG, "device " + std::to_string(d) + ": need nb >= 1, 1 <= bs <= 512, ne >= 0");
    for (int k = 0; k < 8; ++k) L.off[8 * d + k] = acc[k];
    const long long bb = b * b;
    acc[0] += nb * bb;
    acc[1] += (nb - 1) * bb;
    acc[2] += ne;
    acc[3] += ne * bb;
    acc[4] += ne * nb * bb;
    acc[5] += ne * (nb - 1) * bb;
    acc[6] += ne * (nb - 1);
    acc[7] += nb * b;
  }
  for (int k = 0; k < 8; ++k) L.off[8 * (size_t)sys->ndev + k] = acc[k];
  return NEGF_OK;
}

// the host-side work list of the devices `devs` (one block size) of an uneven batch:
// unit u = (device, energy) in device-then-energy order; element offsets of each unit's
// block 0 in the diagonal and off-diagonal outputs; its global energy index
struct WorkList {
  std::vector<int> unit_dev, unit_e, unit_nb, unit_glob;
  std::vector<long long> off_d, off_o;
};

WorkList make_worklist(const negf_system* sys, const Layout& L, const std::vector<int>& devs, long long bb) {
  WorkList w;
  for (size_t k = 0; k < devs.size(); ++k) {
    const int d = devs[k];
    const long long* o = &L.off[8 * (size_t)d];
    const long long nb = sys->nb[d];
    for (int e = 0; e < sys->ne[d]; ++e) {
      w.unit_dev.push_back((int)k);
      w.unit_e.push_back(e);
      w.unit_nb.push_back((int)nb);
      w.unit_glob.push_back((int)(o[2] + e));
      w.off_d.push_back(o[4] + (long long)e * nb * bb);
      w.off_o.push_back(o[5] + (long long)e * (nb - 1) * bb);
    }
  }
  return w;
}

negf_status check_system(Ctx* ctx, const negf_system* sys) {
  if (!sys->H_diag) return fail(ctx, NEGF_ERR_ARG, "H_diag is NULL");
  bool any_multi = false;
  for (int d = 0; d < sys->ndev; ++d) any_multi |= sys->nb[d] > 1;
  if (any_multi && !sys->H_up) return fail(ctx, NEGF_ERR_ARG, "H_up is NULL but some nb > 1");
  if ((sys->S_diag == nullptr) != (sys->S_up == nullptr) && any_multi)
    return fail(ctx, NEGF_ERR_ARG, "S_diag and S_up must both be given or both be NULL");
  if (!sys->energy) return fail(ctx, NEGF_ERR_ARG, "energy is NULL");
  if (!(sys->eta > 0.0) || !isfinite(sys->eta)) return fail(ctx, NEGF_ERR_ARG, "eta must be finite and > 0");
  return NEGF_OK;
}

DevView dev_view(const negf_system* sys, const Layout& L, int d) {
  DevView v;
  const long long* o = &L.off[8 * (size_t)d];
  v.Hd = (const zc*)sys->H_diag + o[0];
  v.Hu = sys->H_up ? (const zc*)sys->H_up + o[1] : nullptr;
  v.Sd = sys->S_diag ? (const zc*)sys->S_diag + o[0] : nullptr;
  v.Su = sys->S_up ? (const zc*)sys->S_up + o[1] : nullptr;
  v.E = sys->energy + o[2];
  v.eta = sys->eta;
  v.nb = sys->nb[d];
  v.b = sys->bs[d];
  return v;
}

ScatView scat_view(const negf_scattering* sc, const Layout& L, int d, int nb, int b) {
  ScatView s{nullptr, nullptr, nullptr, 0};
  if (!sc) return s;
  const long long* o = &L.off[8 * (size_t)d];
  const long long bb = (long long)b * b;
  // block offset of this device: shared => o[0] (sum nb*b*b); per energy => o[4]
  const long long boff = sc->per_energy ? o[4] : o[0];
  s.sigR = sc->sigR ? (const zc*)sc->sigR + boff : nullptr;
  s.sigL = sc->sigL ? (const zc*)sc->sigL + boff : nullptr;
  // scale is [sum ne*nb]: this device starts at sum_{d'<d} ne*nb = sum ne*(nb-1) + sum ne
  s.scale = sc->sigL_scale ? sc->sigL_scale + (o[6] + o[2]) : nullptr;
  s.e_stride = sc->per_energy ? (long long)nb * bb : 0;
  return s;
}

// one device of an uneven batch as the batched sweeps over (device, energy) units see it
struct UnitDev {
  DevView dv;
  ScatView sc;
  const zc *sigma_L, *sigma_R;   // this device's lead blocks (energy 0)
  const double *fL, *fR;         // this device's occupations (energy 0), nullable
};

// ---------------------------------------------------------------------------
// assembly kernels (row a1 of the hot path): blocks of A = z S - H - Sigma and of
// Sigma^< for the units of one step, written to workspace slots
// ---------------------------------------------------------------------------
struct AsmArgs {
  DevView dv;
  ScatView sc;
  int e0;            // first energy (device-local) of the chunk
  int units;
  int i_diag;        // diagonal block index (A_ii and Sigma^<_ii), -1 => none
  int i_off;         // upper block index j (A_{j,j+1} and A_{j+1,j}), -1 => none
  // units are (energy, partition) pairs u = e P + p whose block indices are offset by
  // p L (P = 1: one unit per energy); an off-diagonal index outside [0, nb-1) gives zero
  // blocks
  int P = 1, L = 0;
  // units of an uneven batch: unit u is energy unit_e[u] of device udev[unit_dev[u]]
  // (then dv, sc, e0, the lead pointers and occupations above are unused); a unit whose
  // device has no block i_diag is skipped
  const UnitDev* udev = nullptr;
  const int* unit_dev = nullptr;
  const int* unit_e = nullptr;
  zc *Adiag, *Aup, *Alow, *SigL;   // slot bases (unit stride b*b), each nullable
  zc* SigG;                        // Sigma^>_ii slot (nullable)
  const zc *sigma_L, *sigma_R;     // lead self-energies of this device, [ne] blocks
  const double *fL, *fR;           // this device's occupations (nullable unless SigL)
  // the energy-independent parts of this device's A blocks (asm_w_kernel), nullable:
  // A_ii = E S_ii + Wd_i, A_{j,j+1} = E S_up_j + Wu_j, A_{j+1,j} = (E S_up_j + Wl_j)^H
  // with E real: two FP64 FMAs per element instead of the complex z S - H
  const zc *Wd = nullptr, *Wu = nullptr, *Wl = nullptr;
  // every block index in one launch (grid z = block index k, uniform batches only):
  // A_kk, Sigma^x_kk and A_{k,k+1}, A_{k+1,k} (k < nb-1) into the slot arrays above,
  // block stride units*b*b (i_diag, i_off unused)
  int all_blocks = 0;
};

// Wd_i = -H_ii + i eta S_ii, Wu_j = -H_up_j + i eta S_up_j, Wl_j = -H_up_j - i eta S_up_j
// (then z S - H = E S + W for z = E + i eta, and the conjugate transpose of E S_up + Wl
// is z S_up^H - H_up^H)
__global__ void asm_w_kernel(DevView dv, zc* Wd, zc* Wu, zc* Wl) {
  const int i = blockIdx.y, b = dv.b, nb = dv.nb;
  const int bb = b * b;
  const double eta = dv.eta;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < bb; k += gridDim.x * blockDim.x) {
    const int r = k / b, c = k - r * b;
    const zc sd = dv.Sd ? dv.Sd[(long long)i * bb + k] : zmake(r == c ? 1.0 : 0.0, 0.0);
    const zc hd = dv.Hd[(long long)i * bb + k];
    Wd[(long long)i * bb + k] = zmake(-hd.x - eta * sd.y, -hd.y + eta * sd.x);
    if (i + 1 < nb) {
      const zc su = dv.Su ? dv.Su[(long long)i * bb + k] : zmake(0.0, 0.0);
      const zc hu = dv.Hu[(long long)i * bb + k];
      Wu[(long long)i * bb + k] = zmake(-hu.x - eta * su.y, -hu.y + eta * su.x);
      Wl[(long long)i * bb + k] = zmake(-hu.x + eta * su.y, -hu.y - eta * su.x);
    }
  }
}

// bytes of one device's W blocks (3 nb - 2 blocks, 1 KB aligned)
size_t asm_w_bytes(int nb, int b) {
  return ((sizeof(zc) * (size_t)b * b * (size_t)(3 * nb - 2)) + 1023) & ~(size_t)1023;
}

// One 32 x 32 tile of every requested block per CTA (32 x 8 threads, 4 rows each);
// the conjugate-transposed terms (A_{j+1,j}, the lead Gamma's Sigma^H) are read as the
// transposed tile through shared memory, so that every global access is a row segment.
constexpr int ASM_T = 32;

// USE_W: the E S + W form (a.Wd, a.Wu, a.Wl set); a compile-time switch, so that the
// compiler does not merge the two forms' arithmetic into one predicated sequence
template <bool USE_W>
__global__ void __launch_bounds__(256) assemble_kernel(AsmArgs a) {
  const int u = blockIdx.y;
  int e;
  if (a.udev) {   // the unit's own device
    const UnitDev& D = a.udev[a.unit_dev[u]];
    a.dv = D.dv;
    a.sc = D.sc;
    a.sigma_L = D.sigma_L;
    a.sigma_R = D.sigma_R;
    a.fL = D.fL;
    a.fR = D.fR;
    e = a.unit_e[u];
    if (a.i_diag >= a.dv.nb || a.i_off >= a.dv.nb - 1) return;   // no such block in this device
  } else {
    e = a.e0 + u / a.P;
  }
  const int b = a.dv.b, nb = a.dv.nb;
  const long long bb = (long long)b * b;
  if (a.all_blocks) {
    const int k = blockIdx.z;
    const long long sh = (long long)k * a.units * bb;
    a.i_diag = k;
    a.i_off = (k + 1 < nb) ? k : -1;
    if (a.Adiag) a.Adiag += sh;
    if (a.SigL) a.SigL += sh;
    if (a.SigG) a.SigG += sh;
    if (a.i_off < 0) {
      a.Aup = nullptr;
      a.Alow = nullptr;
    } else {
      if (a.Aup) a.Aup += sh;
      if (a.Alow) a.Alow += sh;
    }
  }
  const int poff = (u % a.P) * a.L;
  const zc z = zmake(a.dv.E[e], a.dv.eta);
  const int ntile = (b + ASM_T - 1) / ASM_T;
  const int r0 = (blockIdx.x / ntile) * ASM_T, c0 = (blockIdx.x % ntile) * ASM_T;
  const int tx = threadIdx.x, ty = threadIdx.y;
  __shared__ zc tS[ASM_T][ASM_T + 1], tH[ASM_T][ASM_T + 1];
  const int i = a.i_diag + poff, j = a.i_off + poff;
  const bool offv = j >= 0 && j < nb - 1;
  const bool lead_lesser = (a.SigL || a.SigG) && (i == 0 || i == nb - 1);
  const zc* sg = (i == 0) ? a.sigma_L + e * bb : a.sigma_R + e * bb;
  const double fo = (i == 0) ? (a.fL ? a.fL[e] : 0.0) : (a.fR ? a.fR[e] : 0.0);
  // transposed tiles: (row c0 + ty + 8k, column r0 + tx) of S_up, H_up (for A_{j+1,j}) and
  // of the lead Sigma (for Sigma^H), stored as [tx][ty + 8k]
  constexpr bool w = USE_W;   // E S + W form (E = Re z)
  const double E = z.x;
  if (a.Alow) {
#pragma unroll
    for (int k = 0; k < ASM_T / 8; ++k) {
      const int rr = c0 + ty + 8 * k, cc = r0 + tx;
      zc sv = zmake(0.0, 0.0), hv = zmake(0.0, 0.0);
      if (rr < b && cc < b && offv) {
        if (a.dv.Su) sv = a.dv.Su[j * bb + (long long)rr * b + cc];
        hv = w ? a.Wl[j * bb + (long long)rr * b + cc] : a.dv.Hu[j * bb + (long long)rr * b + cc];
      }
      tS[tx][ty + 8 * k] = sv;
      tH[tx][ty + 8 * k] = hv;
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < ASM_T / 8; ++k) {
    const int r = r0 + ty + 8 * k, c = c0 + tx;
    if (r >= b || c >= b) continue;
    const long long rc = (long long)r * b + c;
    if (a.Adiag) {
      zc v;
      if (w) {
        const zc wd = a.Wd[i * bb + rc];
        if (a.dv.Sd) {
          const zc sd = a.dv.Sd[i * bb + rc];
          v = zmake(fma(E, sd.x, wd.x), fma(E, sd.y, wd.y));
        } else {
          v = zmake(r == c ? E + wd.x : wd.x, wd.y);
        }
      } else {
        zc sd = a.dv.Sd ? a.dv.Sd[i * bb + rc] : zmake(r == c ? 1.0 : 0.0, 0.0);
        v = zsub(zmul(z, sd), a.dv.Hd[i * bb + rc]);
      }
      if (a.sc.sigR) v = zsub(v, a.sc.sigR[e * a.sc.e_stride + i * bb + rc]);
      if (i == 0) v = zsub(v, a.sigma_L[e * bb + rc]);
      if (i == nb - 1) v = zsub(v, a.sigma_R[e * bb + rc]);
      a.Adiag[u * bb + rc] = v;
    }
    if (a.Aup) {   // A_{j,j+1} = z S_up - H_up
      zc v = zmake(0.0, 0.0);
      if (offv) {
        const zc su = a.dv.Su ? a.dv.Su[j * bb + rc] : zmake(0.0, 0.0);
        if (w) {
          const zc wu = a.Wu[j * bb + rc];
          v = zmake(fma(E, su.x, wu.x), fma(E, su.y, wu.y));
        } else {
          v = zsub(zmul(z, su), a.dv.Hu[j * bb + rc]);
        }
      }
      a.Aup[u * bb + rc] = v;
    }
    if (a.Alow) {  // A_{j+1,j} = z S_up^H - H_up^H: element (r, c) = conj of (c, r)
      const zc st = tS[ty + 8 * k][tx], ht = tH[ty + 8 * k][tx];
      zc v = zmake(0.0, 0.0);
      if (offv) v = w ? zmake(fma(E, st.x, ht.x), fma(-E, st.y, -ht.y)) : zsub(zmul(z, zconj(st)), zconj(ht));
      a.Alow[u * bb + rc] = v;
    }
  }
  if (!a.SigL && !a.SigG) return;
  __syncthreads();
  // transposed tiles: this lead's Sigma (for Sigma^H) and, for Sigma^>, the scattering
  // Sigma^R of block i (for Sigma^A)
  const bool scat_adv = a.SigG && a.sc.sigR;
  if (lead_lesser || scat_adv) {
#pragma unroll
    for (int k = 0; k < ASM_T / 8; ++k) {
      const int rr = c0 + ty + 8 * k, cc = r0 + tx;
      const bool in = rr < b && cc < b;
      if (lead_lesser) tS[tx][ty + 8 * k] = in ? sg[(long long)rr * b + cc] : zmake(0.0, 0.0);
      if (scat_adv)
        tH[tx][ty + 8 * k] = in ? a.sc.sigR[e * a.sc.e_stride + i * bb + (long long)rr * b + cc] : zmake(0.0, 0.0);
    }
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < ASM_T / 8; ++k) {
    const int r = r0 + ty + 8 * k, c = c0 + tx;
    if (r >= b || c >= b) continue;
    const long long rc = (long long)r * b + c;
    zc v = zmake(0.0, 0.0);
    if (a.sc.sigL) {
      const double f = a.sc.scale ? a.sc.scale[(long long)e * nb + i] : 1.0;
      v = zscale(a.sc.sigL[e * a.sc.e_stride + i * bb + rc], f);
    }
    // scattering Sigma^> = Sigma^< + Sigma^R - Sigma^A
    zc vg = v;
    if (scat_adv) vg = zadd(vg, zsub(a.sc.sigR[e * a.sc.e_stride + i * bb + rc], zconj(tH[ty + 8 * k][tx])));
    // lead lesser i f Gamma = -f (Sigma - Sigma^H); lead greater -i (1 - f) Gamma = (1 - f) (Sigma - Sigma^H)
    if (lead_lesser) {
      const zc d = zsub(sg[rc], zconj(tS[ty + 8 * k][tx]));
      v = zsub(v, zscale(d, fo));
      vg = zadd(vg, zscale(d, 1.0 - fo));
      if (nb == 1) {   // both leads on the one block
        const zc* sg2 = a.sigma_R + e * bb;
        const zc d2 = zsub(sg2[rc], zconj(sg2[(long long)c * b + r]));
        const double f2 = a.fR ? a.fR[e] : 0.0;
        v = zsub(v, zscale(d2, f2));
        vg = zadd(vg, zscale(d2, 1.0 - f2));
      }
    }
    if (a.SigL) a.SigL[u * bb + rc] = v;
    if (a.SigG) a.SigG[u * bb + rc] = vg;
  }
}

cudaError_t assemble(const AsmArgs& a, cudaStream_t s) {
  if (a.units <= 0) return cudaSuccess;
  const int nt = (a.dv.b + ASM_T - 1) / ASM_T;
  const dim3 grid((unsigned)(nt * nt), a.units, a.all_blocks ? a.dv.nb : 1);
  if (a.Wd)
    assemble_kernel<true><<<grid, dim3(ASM_T, 8), 0, s>>>(a);
  else
    assemble_kernel<false><<<grid, dim3(ASM_T, 8), 0, s>>>(a);
  return cudaGetLastError();
}

// D = D - W + W^H   (the anti-Hermitian completion of G^<_ii)
__global__ void antiherm_update_kernel(BMat D, BMat W, int n, const int* act) {
  const int u = blockIdx.y;
  if (act && !act[u]) return;
  const long long nn = (long long)n * n;
  zc* d = D.at(u);
  const zc* w = W.at(u);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nn;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / n), c = (int)(idx - (long long)r * n);
    d[idx] = zadd(zsub(d[idx], w[idx]), zconj(w[(long long)c * n + r]));
  }
}

cudaError_t antiherm_update(BMat D, BMat W, int n, int units, cudaStream_t s, const int* act = nullptr) {
  if (units <= 0) return cudaSuccess;
  const long long nn = (long long)n * n;
  dim3 grid((unsigned)std::min<long long>((nn + 255) / 256, 1024), units);
  antiherm_update_kernel<<<grid, 256, 0, s>>>(D, W, n, act);
  return cudaGetLastError();
}

// D = A + B on the masked units
__global__ void add_kernel(BMat D, BMat A, BMat B, int n, const int* act) {
  const int u = blockIdx.y;
  if (act && !act[u]) return;
  const long long nn = (long long)n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x)
    D.at(u)[i] = zadd(A.at(u)[i], B.at(u)[i]);
}

// R = I - R  (R holds M X on entry)
__global__ void one_minus_kernel(BMat R, int n, const int* act) {
  const int u = blockIdx.y;
  if (act && !act[u]) return;
  const long long nn = (long long)n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / n), c = (int)(i - (long long)r * n);
    zc v = R.at(u)[i];
    R.at(u)[i] = zmake((r == c ? 1.0 : 0.0) - v.x, -v.y);
  }
}

// ---------------------------------------------------------------------------
// precision dispatch for the block products
// ---------------------------------------------------------------------------
struct Engine {
  Ctx* ctx;
  cudaStream_t s;
  int mixed;           // 0: FP64, 1: digit-sliced BF16 tensor-core products, 2: TF32 3-term split
  void* inv_scratch;   // for inverses too large for shared memory
  void* oz_scratch = nullptr;   // per-row/column scales of the sliced products (in-kernel digits)
  void* ozt_scratch = nullptr;  // scales and digit images of the digitize-once sliced products
  bool can_slice(int n) const {
    return ozt_scratch ? oz_supported(n) : (oz_scratch != nullptr && oz_inkernel_supported(n));
  }
  // op(A) of the last 8-digit digitize-once product whose scales and digit images are
  // still in the scratch (n <= 128: the kernels whose images cover all of K); any other
  // use of the scratch clears it
  struct AKey {
    const zc* p = nullptr;
    long long us = 0, us2 = 0;
    int inner = 0, opA = 0, n = 0, units = 0, variant = 0;
    const long long* off = nullptr;
    const int* active = nullptr;
    const void* scratch = nullptr;
    bool operator==(const AKey& o) const {
      return p == o.p && us == o.us && us2 == o.us2 && inner == o.inner && opA == o.opA && n == o.n &&
             units == o.units && variant == o.variant && off == o.off && active == o.active && scratch == o.scratch;
    }
  };
  AKey last_a;   // p == nullptr: none
  static AKey key_of(const GemmArgs& g, int variant, const void* scratch) {
    AKey k;
    k.p = g.A.p; k.us = g.A.us; k.us2 = g.A.us2; k.inner = g.A.inner; k.off = g.A.off;
    k.opA = g.opA; k.n = g.n; k.units = g.units; k.active = g.active; k.variant = variant; k.scratch = scratch;
    return k;
  }
  // `reuse`: the caller asks to reuse op(A)'s images when the last product left them
  // (granted only when every field of the operand key matches)
  cudaError_t sliced(GemmArgs g, bool reuse = false) {
    if (!ozt_scratch) {
      last_a = AKey();
      return zgemm_oz(g, oz_scratch, ctx->d_err, s);
    }
    const int v = (g.n >= 0 && g.n <= 512) ? ctx->oz_variant[g.n] : OZ_DEFAULT;
    const int eff = (v == OZ_DEFAULT) ? (g.n <= 96 ? OZ_HALF : g.n <= 128 ? OZ_PERSISTENT : OZ_FULL) : v;
    const AKey k = key_of(g, eff, ozt_scratch);
    const bool keepable = eff != OZ_FULL && g.n <= 128;
    g.reuse_a = (reuse && keepable && last_a.p && last_a == k) ? 1 : 0;
    cudaError_t e = zgemm_ozt_variant(g, ozt_scratch, ctx->d_err, s, v);
    // the images stay valid for the next product unless this one overwrote its own A
    last_a = (e == cudaSuccess && keepable && g.D.p != g.A.p) ? k : AKey();
    return e;
  }
  // a scratch region of the 5-digit product's own (set by the sweeps for their duration),
  // so that its images leave the 8-digit product's in place; without it both share
  // ozt_scratch
  void* ozt_scratch_lo = nullptr;
  cudaError_t sliced_lo(const GemmArgs& g) {
    if (ozt_scratch_lo) return zgemm_ozt_lo(g, ozt_scratch_lo, ctx->d_err, s);
    last_a = AKey();
    return zgemm_ozt_lo(g, ozt_scratch, ctx->d_err, s);
  }
  // timing facility: events around one launch of class `cls`
  int open_cls = -1;
  cudaEvent_t open_ev = nullptr;
  void begin(int cls) {
    ++ctx->launches;
    if (!ctx->prof) return;
    open_cls = cls;
    open_ev = ctx->take_event();
    cudaEventRecord(open_ev, s);
  }
  void end(double flops, double bytes) {
    if (!ctx->prof || open_cls < 0) return;
    cudaEvent_t e1 = ctx->take_event();
    cudaEventRecord(e1, s);
    ctx->recs.push_back(ProfRec{open_cls, open_ev, e1, flops, bytes});
    open_cls = -1;
  }
  // share of the units a masked launch works on, when the caller knows it (the batched
  // sweeps of an uneven batch); < 0: unknown (such launches are counted as "other")
  double active_frac = -1.0;
  // reuse_a: op(A) is the previous product's op(A), unchanged since (see sliced)
  cudaError_t gemm(BMat D, BMat A, int opA, BMat B, int opB, zc alpha, BMat C, zc beta, int n, int units,
                   const int* active = nullptr, bool reuse_a = false) {
    GemmArgs g;
    g.D = D; g.A = A; g.B = B; g.C = C;
    g.opA = opA; g.opB = opB; g.alpha = alpha; g.beta = beta;
    g.n = n; g.units = units; g.active = active;
    const double nn = (double)n * n;
    const double frac = (active && active_frac >= 0.0) ? active_frac : 1.0;
    const double flops = 8.0 * nn * n * units * frac;                        // useful complex flops
    const double bytes = 16.0 * nn * units * frac * (3.0 + (C.p ? 1.0 : 0.0));   // A, B, D (+C) once each
    cudaError_t e;
    const bool masked = active != nullptr && active_frac < 0.0;   // an unknown share of the work
    if (mixed == 1 && can_slice(n)) {
      begin(masked ? K_OTHER : K_GEMM_OZ);
      e = sliced(g, reuse_a);
    } else if (mixed == 2 && tc_supported(n)) {
      begin(masked ? K_OTHER : K_GEMM_TC);
      e = zgemm_tc(g, ctx->d_err, s);
    } else {
      begin(masked ? K_OTHER : K_GEMM_F64);
      e = zgemm_f64(g, s);
    }
    end(masked ? 0.0 : flops, masked ? 0.0 : bytes);
    return e;
  }
  cudaError_t inv(BMat X, BMat M, int n, int units, const int* active, int single, int32_t* status) {
    const bool masked = active != nullptr && active_frac < 0.0;   // an unknown share of the work
    const double frac = (active && active_frac >= 0.0) ? active_frac : 1.0;
    begin(masked ? K_OTHER : (single ? K_INV_F32 : K_INV_F64));
    cudaError_t e = zinv(X, M, n, units, active, single, inv_scratch, status, s);
    end(masked ? 0.0 : 8.0 * (double)n * n * n * units * frac, masked ? 0.0 : 32.0 * (double)n * n * units * frac);
    return e;
  }
  // X = M^{-1}.  Mixed precision: FP32 Gauss-Jordan, then `refine` steps of
  // X <- X + X (I - M X) with the residual I - M X formed in FP64 and the
  // correction product on the engine's GEMM.  T1, T2: scratch slots.
  // Refinement steps: two with the sliced product (each step squares the relative
  // error of the FP32 inverse, so kappa ~ 1e6 blocks need two), one with the TF32 mode.
  cudaError_t inverse(BMat X, BMat M, int n, int units, int32_t* status, BMat T1, BMat T2, int refine = -1,
                      const int* active = nullptr) {
    if (refine < 0) refine = (mixed == 1) ? 2 : 1;
    cudaError_t e = inv(X, M, n, units, active, mixed ? 1 : 0, status);
    if (e != cudaSuccess || !mixed) return e;
    return refine_steps(X, M, n, units, T1, T2, refine, active);
  }
  // `refine` steps X <- X + X (I - M X) (mixed modes); T1 keeps the last residual
  // I - M X (of the X before the last step)
  cudaError_t refine_steps(BMat X, BMat M, int n, int units, BMat T1, BMat T2, int refine, const int* active) {
    cudaError_t e = cudaSuccess;
    const long long nn = (long long)n * n;
    dim3 grid((unsigned)std::min<long long>((nn + 255) / 256, 1024), units);
    for (int k = 0; k < refine; ++k) {
      GemmArgs r;
      r.D = T1; r.A = M; r.B = X; r.C = BMat{nullptr, 0};
      r.opA = OP_N; r.opB = OP_N; r.alpha = zmake(1.0, 0.0); r.beta = zmake(0.0, 0.0);
      r.n = n; r.units = units; r.active = active;
      const double frac = (active && active_frac >= 0.0) ? active_frac : 1.0;
      // I - M X with FP64-class accuracy: the sliced tensor-core product with alpha = -1
      // and the identity added in its epilogue (the same FP64 operation 1 - (M X)_kk),
      // else M X by FP64 FMA and I - M X in a pass of its own
      const bool fused = mixed == 1 && can_slice(n);
      if (fused) {
        r.alpha = zmake(-1.0, 0.0);
        r.plus_identity = 1;
        begin(K_GEMM_OZ);
        // M is the last step's left operand too: its images are reused when the
        // correction in between kept to a scratch region of its own
        e = sliced(r, k > 0);
      } else {
        begin(K_GEMM_F64);
        e = zgemm_f64(r, s);
      }
      end(8.0 * (double)n * n * n * units * frac, 48.0 * (double)n * n * units * frac);
      if (e != cudaSuccess) return e;
      if (!fused) {
        ++ctx->launches;
        one_minus_kernel<<<grid, 256, 0, s>>>(T1, n, active);             // I - M X
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
      }
      if (mixed == 1 && ozt_scratch && oz_supported(n)) {
        // X <- X + X (I - M X) in one product: these kernels read op(A) only through the
        // digit images made before they start, and C and D element by element in one
        // thread, so D, A and C may all be X.  I - M X is small (below ~1e-3 when the
        // FP32 inverse is usable at all), so the correction X (I - M X) needs far less
        // than FP64 class: the 5-digit product (15 slice pairs instead of 36, error
        // ~2^-34 of |X| |I - M X|; 4 digits measured G^R 9e-8 against FP64 at config 2)
        GemmArgs c;
        c.D = X; c.A = X; c.B = T1; c.C = X;
        c.opA = OP_N; c.opB = OP_N; c.alpha = zmake(1.0, 0.0); c.beta = zmake(1.0, 0.0);
        c.n = n; c.units = units; c.active = active;
        const bool masked = active != nullptr && active_frac < 0.0;
        begin(masked ? K_OTHER : K_GEMM_OZ_LO);
        e = sliced_lo(c);
        end(masked ? 0.0 : 8.0 * (double)n * n * n * units * frac, masked ? 0.0 : 64.0 * (double)n * n * units * frac);
        if (e != cudaSuccess) return e;
        continue;
      }
      if ((e = gemm(T2, X, OP_N, T1, OP_N, zmake(1.0, 0.0), BMat{nullptr, 0}, zmake(0.0, 0.0), n, units, active)) !=
          cudaSuccess)
        return e;                                                          // X (I - M X)
      ++ctx->launches;
      add_kernel<<<grid, 256, 0, s>>>(X, X, T2, n, active);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
};

const zc ONE = {1.0, 0.0};
const zc MONE = {-1.0, 0.0};
const zc ZERO = {0.0, 0.0};
const BMat NOMAT = {nullptr, 0};

// ---------------------------------------------------------------------------
// RGF forward/backward sweeps for one device and one chunk of energies
// ---------------------------------------------------------------------------
struct RgfIO {
  const zc *sigma_L, *sigma_R;   // device-offset
  const double *fL, *fR;         // device-offset, nullable for retarded only
  zc *GRd, *GRu, *GRl, *GLd, *GLl;   // device-offset outputs, nullable
  zc *GGd = nullptr, *GGl = nullptr; // device-offset G^> outputs, nullable
  int32_t* status;               // device-offset, nullable
  bool lesser;
  bool greater = false;          // also G^> (with `lesser`)
  const zc* W = nullptr;         // this device's W blocks (asm_w_kernel; Wd, Wu, Wl in turn), nullable
};

// The (device, energy) units of the devices of an uneven batch that share one block size,
// for batched sweeps over all of them (Sec. II: every energy of every device is
// independent): device-side tables in the workspace.  Step i of the forward sweep runs
// on the units whose device has block i, step i of the backward sweep on those with
// block i+1; each launch covers every unit of the group, the others masked out.
struct BatchPlan {
  int nb;                      // the largest block count of the group: the sweeps' length
  const UnitDev* udev;         // [devices of the group]
  const int* unit_dev;         // [U] index into udev
  const int* unit_e;           // [U] device-local energy
  const long long* off_d;      // [U] element offset of the unit's block 0 in GR_diag / GL_diag / GG_diag
  const long long* off_o;      // [U] element offset of the unit's block 0 in the off-diagonal outputs
  const int* act_f;            // [nb][U]: forward step i active (i < nb of the unit's device)
  const int* act_b;            // [nb][U]: backward step i active (i <= nb - 2)
  const double* frac_f;        // host [nb]: share of the units active at forward step i
  const double* frac_b;        // host [nb]: ... at backward step i
  int32_t* st_units;           // [U] per-unit status
};

negf_status rgf_chunk(Ctx* ctx, Engine& eng, const DevView& dv, const ScatView& sc, const RgfIO& io, int e0,
                      int U, char* ws, const BatchPlan* bp = nullptr, int out_e0 = -1) {
  // the output buffers' first block is energy eo's (e0: the caller's full arrays)
  const int eo = out_e0 < 0 ? e0 : out_e0;
  const int nb = bp ? bp->nb : dv.nb, b = dv.b;
  const long long bb = (long long)b * b;
  const size_t blk = sizeof(zc) * bb;
  cudaStream_t s = eng.s;
  // ---- workspace slots (each U blocks, unit stride b*b)
  char* p = ws;
  auto slot = [&](int count) { zc* q = (zc*)p; p += blk * (size_t)U * count; return q; };
  // small blocks: the whole sweep in one launch over blocks assembled for every index
  const bool small = !bp && rgf_small_supported(b, eng.mixed);
  const int nd = small ? nb : 1, no = small ? std::max(nb - 1, 1) : 1;
  zc* Adiag = slot(nd);
  zc* Aup = slot(no);
  zc* Alow = slot(no);
  zc* SigL = io.lesser ? slot(nd) : nullptr;
  const bool greater = io.lesser && io.greater;
  zc* SigG = greater ? slot(nd) : nullptr;
  zc* T[4];
  for (int k = 0; k < 4; ++k) T[k] = slot(1);
  zc* Ybase = slot(std::max(nb - 1, 1));
  zc* gbase = io.GRd ? nullptr : slot(nb);
  zc* glbase = (io.lesser && !io.GLd) ? slot(nb) : nullptr;
  zc* ggbase = (greater && !io.GGd) ? slot(nb) : nullptr;
  zc* gup_tmp = io.GRu ? nullptr : slot(1);
  if (zinv_scratch_bytes(b, U, eng.mixed ? 1 : 0) > 0) {
    eng.inv_scratch = (void*)p;
    p += zinv_scratch_bytes(b, U, eng.mixed ? 1 : 0);
  }
  p = (char*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
  eng.ozt_scratch = (void*)p;
  // the 5-digit correction products in a region of their own for the duration of the
  // sweeps (the refinement's residuals then reuse M's images)
  struct LoScratch {
    Engine& e;
    ~LoScratch() { e.ozt_scratch_lo = nullptr; }
  } lo_guard{eng};
  if (eng.mixed == 1 && oz_supported(b))
    eng.ozt_scratch_lo = (void*)(p + ((ozt_scratch_bytes(b, U) + 1023) & ~(size_t)1023));

  auto S1 = [&](zc* base) { return BMat{base, bb}; };
  // per-energy output blocks: [e][i] with unit stride nb*b*b (diag) or (nb-1)*b*b (off-diagonal);
  // for an uneven batch, block i of unit u at base + off[u] + i b*b
  auto outD = [&](zc* base, int i) {
    if (bp) return BMat{base + (long long)i * bb, 0, 0, 0, bp->off_d};
    return BMat{base + ((long long)(e0 - eo) * nb + i) * bb, (long long)nb * bb};
  };
  auto gD = [&](int i) { return io.GRd ? outD(io.GRd, i) : BMat{gbase + (long long)i * U * bb, bb}; };
  auto glD = [&](int i) { return io.GLd ? outD(io.GLd, i) : BMat{glbase + (long long)i * U * bb, bb}; };
  auto ggD = [&](int i) { return io.GGd ? outD(io.GGd, i) : BMat{ggbase + (long long)i * U * bb, bb}; };
  auto Yb = [&](int i) { return BMat{Ybase + (long long)i * U * bb, bb}; };
  // the Keldysh kinds of this call: G^< and, with `greater`, G^> (the same recursion on
  // Sigma^> in place of Sigma^<)
  struct Kind { zc* sig; std::function<BMat(int)> D; zc* low; };
  std::vector<Kind> kinds;
  if (io.lesser) kinds.push_back(Kind{SigL, glD, io.GLl});
  if (greater) kinds.push_back(Kind{SigG, ggD, io.GGl});
  auto offB = [&](zc* base, int i) {
    if (bp) return BMat{base + (long long)i * bb, 0, 0, 0, bp->off_o};
    return BMat{base + ((long long)(e0 - eo) * (nb - 1) + i) * bb, (long long)(nb - 1) * bb};
  };

  AsmArgs a;
  a.dv = dv; a.sc = sc; a.e0 = e0; a.units = U;
  a.sigma_L = io.sigma_L; a.sigma_R = io.sigma_R; a.fL = io.fL; a.fR = io.fR;
  if (bp) { a.udev = bp->udev; a.unit_dev = bp->unit_dev; a.unit_e = bp->unit_e; }
  if (io.W && !bp) {
    a.Wd = io.W;
    a.Wu = io.W + (long long)nb * bb;
    a.Wl = a.Wu + (long long)(nb - 1) * bb;
  }
  int32_t* st = bp ? bp->st_units : (io.status ? io.status + e0 : nullptr);
  const int* act = nullptr;   // this step's mask (uneven batch), else every unit

  if (small) {
    a.all_blocks = 1;
    a.Adiag = Adiag; a.SigL = SigL; a.SigG = SigG;
    a.Aup = nb > 1 ? Aup : nullptr;
    a.Alow = nb > 1 ? Alow : nullptr;
    ++ctx->launches;
    CU(assemble(a, s));
    const SBlk none{nullptr, 0, 0};
    // an output array [e][i] from energy e0 on, else a workspace slot array [i][u]
    auto diag = [&](zc* out, zc* w) {
      return out ? SBlk{out + (long long)(e0 - eo) * nb * bb, (long long)nb * bb, bb} : SBlk{w, bb, (long long)U * bb};
    };
    auto offd = [&](zc* out) {
      return out ? SBlk{out + (long long)(e0 - eo) * (nb - 1) * bb, (long long)(nb - 1) * bb, bb} : none;
    };
    SmallSweep w;
    w.nb = nb; w.b = b; w.U = U; w.nk = (int)kinds.size();
    w.Ad = Adiag; w.Au = Aup; w.Al = Alow; w.Sl = SigL; w.Sg = SigG;
    w.Y = SBlk{Ybase, bb, (long long)U * bb};
    w.gR = diag(io.GRd, gbase);
    w.gL = io.lesser ? diag(io.GLd, glbase) : none;
    w.gG = greater ? diag(io.GGd, ggbase) : none;
    w.Ru = offd(io.GRu);
    w.Rl = offd(io.GRl);
    w.Ll = io.lesser ? offd(io.GLl) : none;
    w.Gl = greater ? offd(io.GGl) : none;
    w.status = st;
    // useful work: nb inverses, the retarded products (2 per forward step, 3 or 4 per
    // backward step) and per Keldysh kind 2 + 4 (nb - 1) forward and 4 or 5 per backward step
    const int nk = w.nk, m = nb - 1;
    const double prods = 2.0 * m + m * (3.0 + (io.GRl ? 1 : 0)) +
                         nk * (2.0 + 4.0 * m + m * (4.0 + (io.GLl ? 1 : 0)));
    const double blocks = nb * (5.0 + 2 * nk) + m * (5.0 + (io.GRu ? 1 : 0) + (io.GRl ? 1 : 0) + nk * 3.0);
    eng.begin(K_GEMM_F64);
    CU(rgf_small_sweep(w, s));
    eng.end(8.0 * bb * b * (prods + nb) * U, 16.0 * bb * blocks * U);
    return NEGF_OK;
  }

  // ---------------- forward sweep
  for (int i = 0; i < nb; ++i) {
    if (bp) { act = bp->act_f + (size_t)i * U; eng.active_frac = bp->frac_f[i]; }
    a.i_diag = i;
    a.i_off = i - 1;
    a.Adiag = Adiag; a.SigL = SigL; a.SigG = SigG;
    a.Aup = (i > 0) ? Aup : nullptr;
    a.Alow = (i > 0) ? Alow : nullptr;
    ++ctx->launches;
    CU(assemble(a, s));
    if (i == 0) {
      CU(eng.inverse(gD(0), S1(Adiag), b, U, st, S1(T[1]), S1(T[2]), -1, act));
      for (const Kind& k : kinds) {
        CU(eng.gemm(S1(T[2]), gD(0), OP_N, S1(k.sig), OP_N, ONE, NOMAT, ZERO, b, U, act));
        CU(eng.gemm(k.D(0), S1(T[2]), OP_N, gD(0), OP_H, ONE, NOMAT, ZERO, b, U, act));
      }
      continue;
    }
    // Y_{i-1} = A_{i,i-1} g_{i-1};  M = A_ii - Y_{i-1} A_{i-1,i};  g_i = M^{-1}.  The first
    // Keldysh kind's A_{i,i-1} g^x_{i-1} right after Y (the same left operand: the sliced
    // product keeps its digit images), into T3, which the inverse leaves alone
    CU(eng.gemm(Yb(i - 1), S1(Alow), OP_N, gD(i - 1), OP_N, ONE, NOMAT, ZERO, b, U, act));
    if (!kinds.empty())
      CU(eng.gemm(S1(T[3]), S1(Alow), OP_N, kinds[0].D(i - 1), OP_N, ONE, NOMAT, ZERO, b, U, act, true));
    CU(eng.gemm(S1(T[0]), Yb(i - 1), OP_N, S1(Aup), OP_N, MONE, S1(Adiag), ONE, b, U, act));
    CU(eng.inverse(gD(i), S1(T[0]), b, U, st, S1(T[1]), S1(T[2]), -1, act));
    for (size_t x = 0; x < kinds.size(); ++x) {
      const Kind& k = kinds[x];
      // g^x_i = g_i (Sigma^x_ii + A_{i,i-1} g^x_{i-1} A_{i,i-1}^H) g_i^H   (x = <, >)
      const BMat T1 = S1(x == 0 ? T[3] : T[1]), T3 = S1(x == 0 ? T[1] : T[3]);
      if (x > 0) CU(eng.gemm(T1, S1(Alow), OP_N, k.D(i - 1), OP_N, ONE, NOMAT, ZERO, b, U, act));
      CU(eng.gemm(S1(T[2]), T1, OP_N, S1(Alow), OP_H, ONE, S1(k.sig), ONE, b, U, act));
      CU(eng.gemm(T3, gD(i), OP_N, S1(T[2]), OP_N, ONE, NOMAT, ZERO, b, U, act));
      CU(eng.gemm(k.D(i), T3, OP_N, gD(i), OP_H, ONE, NOMAT, ZERO, b, U, act));
    }
  }
  // ---------------- backward sweep
  a.Adiag = nullptr; a.SigL = nullptr; a.SigG = nullptr;
  for (int i = nb - 2; i >= 0; --i) {
    if (bp) { act = bp->act_b + (size_t)i * U; eng.active_frac = bp->frac_b[i]; }
    a.i_diag = -1;
    a.i_off = i;
    a.Aup = Aup; a.Alow = Alow;
    ++ctx->launches;
    CU(assemble(a, s));
    const BMat X = S1(T[0]);
    const BMat Gup = io.GRu ? offB(io.GRu, i) : S1(gup_tmp);
    // X = g_i A_{i,i+1};  G_{i,i+1} = -X G_{i+1,i+1};  G_ii = g_i - G_{i,i+1} Y_i;  G_{i+1,i} = -G_{i+1,i+1} Y_i;
    // per Keldysh kind x = <, >:  Z = A_{i+1,i} g^x_i,  P = G^x_{i+1,i+1} X^H,  W = G_{i,i+1} Z,
    // G^x_ii = g^x_i + X P - W + W^H,  G^x_{i+1,i} = -G_{i+1,i+1} Z - P.
    // The first kind's products are ordered so that the pairs with the same left operand
    // (X; G_{i,i+1}; G_{i+1,i+1}) run back to back: the sliced product keeps that
    // operand's digit images for the second of each pair
    CU(eng.gemm(X, gD(i), OP_N, S1(Aup), OP_N, ONE, NOMAT, ZERO, b, U, act));
    const Kind* k0 = kinds.empty() ? nullptr : &kinds[0];
    const BMat Z = S1(T[1]), P = S1(T[2]), Wm = S1(T[3]);
    if (k0) {
      CU(eng.gemm(Z, S1(Alow), OP_N, k0->D(i), OP_N, ONE, NOMAT, ZERO, b, U, act));
      CU(eng.gemm(P, k0->D(i + 1), OP_N, X, OP_H, ONE, NOMAT, ZERO, b, U, act));
    }
    CU(eng.gemm(Gup, X, OP_N, gD(i + 1), OP_N, MONE, NOMAT, ZERO, b, U, act));
    if (k0) CU(eng.gemm(k0->D(i), X, OP_N, P, OP_N, ONE, k0->D(i), ONE, b, U, act, true));
    CU(eng.gemm(gD(i), Gup, OP_N, Yb(i), OP_N, MONE, gD(i), ONE, b, U, act));
    if (k0) {
      CU(eng.gemm(Wm, Gup, OP_N, Z, OP_N, ONE, NOMAT, ZERO, b, U, act, true));
      ++ctx->launches;
      CU(antiherm_update(k0->D(i), Wm, b, U, s, act));
    }
    if (io.GRl) CU(eng.gemm(offB(io.GRl, i), gD(i + 1), OP_N, Yb(i), OP_N, MONE, NOMAT, ZERO, b, U, act));
    if (k0 && k0->low)
      CU(eng.gemm(offB(k0->low, i), gD(i + 1), OP_N, Z, OP_N, MONE, P, MONE, b, U, act, io.GRl != nullptr));
    for (size_t x = 1; x < kinds.size(); ++x) {
      const Kind& k = kinds[x];
      CU(eng.gemm(Z, S1(Alow), OP_N, k.D(i), OP_N, ONE, NOMAT, ZERO, b, U, act));
      CU(eng.gemm(P, k.D(i + 1), OP_N, X, OP_H, ONE, NOMAT, ZERO, b, U, act));
      CU(eng.gemm(Wm, Gup, OP_N, Z, OP_N, ONE, NOMAT, ZERO, b, U, act));
      CU(eng.gemm(k.D(i), X, OP_N, P, OP_N, ONE, k.D(i), ONE, b, U, act));
      ++ctx->launches;
      CU(antiherm_update(k.D(i), Wm, b, U, s, act));
      if (k.low) CU(eng.gemm(offB(k.low, i), gD(i + 1), OP_N, Z, OP_N, MONE, P, MONE, b, U, act));
    }
  }
  eng.active_frac = -1.0;
  return NEGF_OK;
}

// dst[u] = src[u] (units of any BMat layout)
__global__ void bcopy_kernel(BMat dst, BMat src, int n) {
  const int u = blockIdx.y;
  const long long nn = (long long)n * n;
  zc* d = dst.at(u);
  const zc* q = src.at(u);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x)
    d[i] = q[i];
}

cudaError_t bcopy(BMat dst, BMat src, int n, int units, cudaStream_t s) {
  if (units <= 0) return cudaSuccess;
  const long long nn = (long long)n * n;
  bcopy_kernel<<<dim3((unsigned)std::min<long long>((nn + 255) / 256, 1024), units), 256, 0, s>>>(dst, src, n);
  return cudaGetLastError();
}

// status[e] = the worst (most negative) code of the units e*P .. e*P+P-1
__global__ void status_merge_kernel(int32_t* status, const int32_t* st_units, int U, int P) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= U) return;
  int32_t w = status[e];
  for (int p = 0; p < P; ++p) w = min(w, st_units[(long long)e * P + p]);
  status[e] = w;
}

// ---------------------------------------------------------------------------
// partitioned selected inversion of G^R (Sec. II, Fig. 3): P partitions of L = nb/P
// blocks, one unit per (energy, partition) u = e P + p, so that every step is one
// batched launch over U P units.  Partition p eliminates its interior blocks
// pL .. pL+L-2 downward with the previous partition's last block e_(p-1) = pL-1 as the
// top boundary a and its own last block e_p = pL+L-1 as the bottom boundary b:
//   g_k = D_k^{-1};  Y_k = A_ji g_k, X_k = g_k A_ij, Xa_k = F_ak g_k, Wa_k = g_k F_ka;
//   D_j = A_jj - Y_k A_ij, F_aj = -Xa_k A_ij, F_ja = -Y_k F_ka, dD_a -= Xa_k F_ka
// (F = 0 for p = 0).  The boundaries e_0 .. e_(P-1) form a BT system with diagonal
// D_(e_r) + dD_a of partition r+1 and couplings F_ab, F_ba of partition r+1, inverted
// by the block recursion (one unit per energy).  Each partition then rebuilds its
// interior from the boundary blocks of G, k = L-2 .. 0, j = k+1:
//   G_jk = -(G_ja Xa_k + G_jj Y_k), G_ak = -(G_aa Xa_k + G_aj Y_k),
//   G_kj = -(Wa_k G_aj + X_k G_jj), G_ka = -(Wa_k G_aa + X_k G_ja),
//   G_kk = g_k - (Wa_k G_ak + X_k G_jk),
// and G_(a,pL), G_(pL,a) are the off-diagonal blocks between partitions.
// ---------------------------------------------------------------------------
size_t partitioned_bytes_per_energy(int nb, int b, int P, int mixed) {
  const int L = nb / P;
  const size_t blk = sizeof(zc) * (size_t)b * b;
  // per (energy, partition): 17 working slots + 4 (L - 1) stored factors; per energy:
  // 2 (P - 1) reduced-recursion slots + 1; per unit status word
  size_t bytes = blk * ((size_t)P * (17 + 4 * (size_t)(L - 1)) + 2 * (size_t)std::max(P - 1, 1) + 1);
  bytes += sizeof(int32_t) * (size_t)P + 256;
  bytes += zinv_scratch_bytes(b, P, mixed ? 1 : 0);
  if (mixed == 1) bytes += ozt_scratch_bytes(b, P) + 1024;
  return bytes;
}

negf_status rgf_partitioned_chunk(Ctx* ctx, Engine& eng, const DevView& dv, const ScatView& sc, const RgfIO& io,
                                  int P, int e0, int U, char* ws) {
  const int nb = dv.nb, b = dv.b, L = nb / P, UP = U * P;
  const long long bb = (long long)b * b;
  const size_t blk = sizeof(zc) * bb;
  cudaStream_t s = eng.s;
  char* p = ws;
  auto slots = [&](long long count) { zc* q = (zc*)p; p += blk * (size_t)count; return q; };
  auto S1 = [&](zc* base) { return BMat{base, bb}; };
  zc *Adiag = slots(UP), *Aup = slots(UP), *Alow = slots(UP), *D = slots(UP), *dDa = slots(UP);
  zc *Fak = slots(UP), *Fka = slots(UP), *Fak2 = slots(UP), *Fka2 = slots(UP);
  zc *T0 = slots(UP), *T1 = slots(UP), *T2 = slots(UP);
  zc *Gaa = slots(UP), *Gaj = slots(UP), *Gja = slots(UP), *Gak = slots(UP), *Gka = slots(UP);
  zc* Yf = slots((long long)UP * (L - 1));
  zc* Xf = slots((long long)UP * (L - 1));
  zc* Xaf = slots((long long)UP * (L - 1));
  zc* Waf = slots((long long)UP * (L - 1));
  zc* RY = slots((long long)U * std::max(P - 1, 1));   // reduced recursion: A_(r+1,r) g_r per energy
  zc* RX = slots(U);
  int32_t* st_units = (int32_t*)p;
  p += ((sizeof(int32_t) * (size_t)UP + 255) / 256) * 256;
  if (zinv_scratch_bytes(b, UP, eng.mixed ? 1 : 0) > 0) {
    eng.inv_scratch = (void*)p;
    p += zinv_scratch_bytes(b, UP, eng.mixed ? 1 : 0);
  }
  p = (char*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
  eng.ozt_scratch = (void*)p;

  // outputs seen per (energy, partition) unit: block pL + k of energy e0 + e
  auto outD = [&](int k) { return BMat{io.GRd + ((long long)e0 * nb + k) * bb, (long long)nb * bb, P, L * bb}; };
  auto outU = [&](zc* base, int k) {
    return BMat{base + ((long long)e0 * (nb - 1) + k) * bb, (long long)(nb - 1) * bb, P, L * bb};
  };
  auto fac = [&](zc* base, int k) { return BMat{base + (long long)k * UP * bb, bb}; };
  // per energy, the entry of partition r of a [U P] slot
  auto ofP = [&](zc* base, int r) { return BMat{base + (long long)r * bb, (long long)P * bb}; };
  // per energy, the output block e_r = rL + L - 1
  auto redD = [&](int r) { return BMat{io.GRd + ((long long)e0 * nb + (long long)r * L + L - 1) * bb, (long long)nb * bb}; };
  auto RYb = [&](int r) { return BMat{RY + (long long)r * U * bb, bb}; };

  CU(cudaMemsetAsync(st_units, 0, sizeof(int32_t) * (size_t)UP, s));
  AsmArgs a;
  a.dv = dv; a.sc = sc; a.e0 = e0; a.units = UP; a.P = P; a.L = L;
  a.sigma_L = io.sigma_L; a.sigma_R = io.sigma_R; a.fL = nullptr; a.fR = nullptr;
  a.SigL = nullptr; a.SigG = nullptr;
  // ---------------- elimination of the interiors, all partitions at once
  a.i_diag = 0; a.i_off = -1;                    // D_0 = A_(pL,pL); F_a0, F_0a = A_(pL-1,pL), A_(pL,pL-1)
  a.Adiag = D; a.Aup = Fak; a.Alow = Fka;
  ++ctx->launches;
  CU(assemble(a, s));
  CU(cudaMemsetAsync(dDa, 0, blk * (size_t)UP, s));
  for (int k = 0; k + 1 < L; ++k) {
    CU(eng.inverse(outD(k), S1(D), b, UP, st_units, S1(T1), S1(T2)));      // g_k (in the G_kk output)
    a.i_diag = k + 1; a.i_off = k;
    a.Adiag = Adiag; a.Aup = Aup; a.Alow = Alow;
    ++ctx->launches;
    CU(assemble(a, s));                                                     // A_jj, A_ij, A_ji
    CU(eng.gemm(fac(Yf, k), S1(Alow), OP_N, outD(k), OP_N, ONE, NOMAT, ZERO, b, UP));
    CU(eng.gemm(fac(Xf, k), outD(k), OP_N, S1(Aup), OP_N, ONE, NOMAT, ZERO, b, UP));
    CU(eng.gemm(fac(Xaf, k), S1(Fak), OP_N, outD(k), OP_N, ONE, NOMAT, ZERO, b, UP));
    CU(eng.gemm(fac(Waf, k), outD(k), OP_N, S1(Fka), OP_N, ONE, NOMAT, ZERO, b, UP));
    CU(eng.gemm(S1(D), fac(Yf, k), OP_N, S1(Aup), OP_N, MONE, S1(Adiag), ONE, b, UP));      // D_j
    CU(eng.gemm(S1(dDa), fac(Xaf, k), OP_N, S1(Fka), OP_N, MONE, S1(dDa), ONE, b, UP));     // dD_a
    CU(eng.gemm(S1(Fak2), fac(Xaf, k), OP_N, S1(Aup), OP_N, MONE, NOMAT, ZERO, b, UP));     // F_aj
    CU(eng.gemm(S1(Fka2), fac(Yf, k), OP_N, S1(Fka), OP_N, MONE, NOMAT, ZERO, b, UP));      // F_ja
    std::swap(Fak, Fak2);
    std::swap(Fka, Fka2);
  }
  // ---------------- the reduced BT system over the boundaries, one unit per energy
  int32_t* st = io.status ? io.status + e0 : nullptr;
  for (int r = 0; r < P; ++r) {
    BMat M = ofP(D, r);
    if (r + 1 < P) {                                                        // + dD_a of partition r+1
      ++ctx->launches;
      const long long nn = bb;
      add_kernel<<<dim3((unsigned)std::min<long long>((nn + 255) / 256, 1024), U), 256, 0, s>>>(
          S1(T0), ofP(D, r), ofP(dDa, r + 1), b, nullptr);
      CU(cudaGetLastError());
      M = S1(T0);
    }
    if (r > 0)                                                              // - A_(r,r-1) g_(r-1) A_(r-1,r)
      CU(eng.gemm(S1(T0), RYb(r - 1), OP_N, ofP(Fak, r), OP_N, MONE, M, ONE, b, U));
    CU(eng.inverse(redD(r), (r > 0 || r + 1 < P) ? S1(T0) : M, b, U, st, S1(T1), S1(T2)));
    if (r + 1 < P) CU(eng.gemm(RYb(r), ofP(Fka, r + 1), OP_N, redD(r), OP_N, ONE, NOMAT, ZERO, b, U));
  }
  // G_aa, G_ab, G_ba of partition p (= G at e_(p-1), G_(e_(p-1), e_p), G_(e_p, e_(p-1))); zero for p = 0
  CU(cudaMemsetAsync(Gaa, 0, blk * (size_t)UP, s));
  CU(cudaMemsetAsync(Gaj, 0, blk * (size_t)UP, s));
  CU(cudaMemsetAsync(Gja, 0, blk * (size_t)UP, s));
  for (int r = P - 2; r >= 0; --r) {
    // X = g_r A_(r,r+1); G_(r,r+1) = -X G_(r+1,r+1); G_(r+1,r) = -G_(r+1,r+1) Y_r; G_rr = g_r - G_(r,r+1) Y_r
    CU(eng.gemm(S1(RX), redD(r), OP_N, ofP(Fak, r + 1), OP_N, ONE, NOMAT, ZERO, b, U));
    CU(eng.gemm(ofP(Gaj, r + 1), S1(RX), OP_N, redD(r + 1), OP_N, MONE, NOMAT, ZERO, b, U));
    CU(eng.gemm(ofP(Gja, r + 1), redD(r + 1), OP_N, RYb(r), OP_N, MONE, NOMAT, ZERO, b, U));
    CU(eng.gemm(redD(r), ofP(Gaj, r + 1), OP_N, RYb(r), OP_N, MONE, redD(r), ONE, b, U));
    ++ctx->launches;
    CU(bcopy(ofP(Gaa, r + 1), redD(r), b, U, s));
  }
  // ---------------- reconstruction of the interiors, all partitions at once
  zc* GRu = io.GRu;
  zc* GRl = io.GRl;
  for (int k = L - 2; k >= 0; --k) {
    const BMat Gjj = outD(k + 1);
    // G_jk = -(G_ja Xa_k) - G_jj Y_k
    CU(eng.gemm(S1(T0), S1(Gja), OP_N, fac(Xaf, k), OP_N, ONE, NOMAT, ZERO, b, UP));
    CU(eng.gemm(outU(GRl, k), Gjj, OP_N, fac(Yf, k), OP_N, MONE, S1(T0), MONE, b, UP));
    // G_ak = -(G_aa Xa_k) - G_aj Y_k
    CU(eng.gemm(S1(T0), S1(Gaa), OP_N, fac(Xaf, k), OP_N, ONE, NOMAT, ZERO, b, UP));
    CU(eng.gemm(S1(Gak), S1(Gaj), OP_N, fac(Yf, k), OP_N, MONE, S1(T0), MONE, b, UP));
    // G_kj = -(Wa_k G_aj) - X_k G_jj
    CU(eng.gemm(S1(T0), fac(Waf, k), OP_N, S1(Gaj), OP_N, ONE, NOMAT, ZERO, b, UP));
    CU(eng.gemm(outU(GRu, k), fac(Xf, k), OP_N, Gjj, OP_N, MONE, S1(T0), MONE, b, UP));
    // G_ka = -(Wa_k G_aa) - X_k G_ja
    CU(eng.gemm(S1(T0), fac(Waf, k), OP_N, S1(Gaa), OP_N, ONE, NOMAT, ZERO, b, UP));
    CU(eng.gemm(S1(Gka), fac(Xf, k), OP_N, S1(Gja), OP_N, MONE, S1(T0), MONE, b, UP));
    // G_kk = g_k - Wa_k G_ak - X_k G_jk   (in place over g_k)
    CU(eng.gemm(outD(k), fac(Waf, k), OP_N, S1(Gak), OP_N, MONE, outD(k), ONE, b, UP));
    CU(eng.gemm(outD(k), fac(Xf, k), OP_N, outU(GRl, k), OP_N, MONE, outD(k), ONE, b, UP));
    std::swap(Gaj, Gak);
    std::swap(Gja, Gka);
  }
  // the blocks between partitions: (pL-1, pL) = G_(a,pL), (pL, pL-1) = G_(pL,a), p >= 1
  if (P > 1) {
    const BMat dstU{GRu + ((long long)e0 * (nb - 1) + L - 1) * bb, (long long)(nb - 1) * bb, P - 1, L * bb};
    const BMat dstL{GRl + ((long long)e0 * (nb - 1) + L - 1) * bb, (long long)(nb - 1) * bb, P - 1, L * bb};
    const BMat srcU{Gaj + bb, (long long)P * bb, P - 1, bb};
    const BMat srcL{Gja + bb, (long long)P * bb, P - 1, bb};
    ctx->launches += 2;
    CU(bcopy(dstU, srcU, b, U * (P - 1), s));
    CU(bcopy(dstL, srcL, b, U * (P - 1), s));
  }
  if (st) {
    ++ctx->launches;
    status_merge_kernel<<<(U + 127) / 128, 128, 0, s>>>(st, st_units, U, P);
    CU(cudaGetLastError());
  }
  return NEGF_OK;
}

// ---------------------------------------------------------------------------
// arrowhead BT (BTA): the device's BT matrix bordered by a tip block t (a gate, size b,
// overlap I) coupled to every block: A_tt = z I - H_tip, A_(t,i) = -H_(t,i),
// A_(i,t) = -H_(t,i)^H.  All device blocks are eliminated downward with the tip as the
// boundary every block couples to (the partitioned recursions with a = t, plus the
// arrow's own coupling at every block):
//   D_0 = A_00, F_t0 = A_t0, F_0t = A_0t;  g_k = D_k^{-1}, Xt_k = F_tk g_k, Wt_k = g_k F_kt,
//   dD_t -= Xt_k F_kt;  for j = k+1: Y_k = A_jk g_k, X_k = g_k A_kj, D_j = A_jj - Y_k A_kj,
//   F_tj = A_tj - Xt_k A_kj, F_jt = A_jt - Y_k F_kt;
// then G_tt = (A_tt + dD_t)^{-1}, and from the last block up:
//   G_tk = -(G_tt Xt_k + G_tj Y_k),  G_kt = -(Wt_k G_tt + X_k G_jt),
//   G_jk = -(G_jt Xt_k + G_jj Y_k),  G_kj = -(Wt_k G_tj + X_k G_jj),
//   G_kk = g_k - (Wt_k G_tk + X_k G_jk)      (the j terms absent for the last block).
// ---------------------------------------------------------------------------
__global__ void tip_assemble_kernel(BMat Att, const zc* H_tip, const double* E, double eta, int e0, int n) {
  const int u = blockIdx.y;
  const zc z = zmake(E[e0 + u], eta);
  const long long nn = (long long)n * n;
  zc* d = Att.at(u);
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nn; k += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(k / n), c = (int)(k - (long long)r * n);
    zc v = zmake(-H_tip[k].x, -H_tip[k].y);
    if (r == c) v = zadd(v, z);
    d[k] = v;
  }
}

// the arrow's blocks of A, shared by all energies: row[i] = -H_(t,i), col[i] = -H_(t,i)^H
__global__ void arrow_blocks_kernel(zc* row, zc* col, const zc* H, int n) {
  const int i = blockIdx.y;
  const long long nn = (long long)n * n;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < nn; k += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(k / n), c = (int)(k - (long long)r * n);
    const zc h = H[(long long)i * nn + k];
    const zc ht = H[(long long)i * nn + (long long)c * n + r];
    row[(long long)i * nn + k] = zmake(-h.x, -h.y);
    col[(long long)i * nn + k] = zmake(-ht.x, ht.y);
  }
}

struct ArrowIO {
  const zc* H_tip;     // this device's tip Hamiltonian
  const zc* H_arrow;   // this device's [nb] blocks H_(t,i)
  zc *Gt, *Grow, *Gcol;   // device-offset outputs: [ne] tip blocks, [ne][nb] G_(t,i), G_(i,t)
};

size_t arrowhead_bytes_per_energy(int nb, int b, int mixed) {
  const size_t blk = sizeof(zc) * (size_t)b * b;
  size_t bytes = blk * (13 + 4 * (size_t)nb);
  bytes += zinv_scratch_bytes(b, 1, mixed ? 1 : 0);
  if (mixed == 1) bytes += ozt_scratch_bytes(b, 1) + 1024;
  return bytes;
}

// Arow, Acol: the device's shared arrow blocks of A (arrow_blocks_kernel)
negf_status rgf_arrowhead_chunk(Ctx* ctx, Engine& eng, const DevView& dv, const ScatView& sc, const RgfIO& io,
                                const ArrowIO& ar, const zc* Arow, const zc* Acol, int e0, int U, char* ws) {
  const int nb = dv.nb, b = dv.b;
  const long long bb = (long long)b * b;
  const size_t blk = sizeof(zc) * bb;
  cudaStream_t s = eng.s;
  char* p = ws;
  auto slots = [&](long long count) { zc* q = (zc*)p; p += blk * (size_t)count; return q; };
  auto S1 = [&](zc* base) { return BMat{base, bb}; };
  zc *Adiag = slots(U), *Aup = slots(U), *Alow = slots(U), *D = slots(U), *dDt = slots(U);
  zc *Ft = slots(U), *Fc = slots(U), *Ft2 = slots(U), *Fc2 = slots(U);
  zc *T0 = slots(U), *T1 = slots(U), *T2 = slots(U), *Att = slots(U);
  zc* Yf = slots((long long)U * nb);
  zc* Xf = slots((long long)U * nb);
  zc* Xtf = slots((long long)U * nb);
  zc* Wtf = slots((long long)U * nb);
  if (zinv_scratch_bytes(b, U, eng.mixed ? 1 : 0) > 0) {
    eng.inv_scratch = (void*)p;
    p += zinv_scratch_bytes(b, U, eng.mixed ? 1 : 0);
  }
  p = (char*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
  eng.ozt_scratch = (void*)p;
  auto outD = [&](int k) { return BMat{io.GRd + ((long long)e0 * nb + k) * bb, (long long)nb * bb}; };
  auto offB = [&](zc* base, int k) { return BMat{base + ((long long)e0 * (nb - 1) + k) * bb, (long long)(nb - 1) * bb}; };
  auto arr = [&](zc* base, int k) { return BMat{base + ((long long)e0 * nb + k) * bb, (long long)nb * bb}; };
  auto fac = [&](zc* base, int k) { return BMat{base + (long long)k * U * bb, bb}; };
  auto shared = [&](const zc* base, int k) { return BMat{(zc*)base + (long long)k * bb, 0}; };
  const BMat Gtt{ar.Gt + (long long)e0 * bb, bb};
  int32_t* st = io.status ? io.status + e0 : nullptr;
  const dim3 eg((unsigned)std::min<long long>((bb + 255) / 256, 1024), U);

  AsmArgs a;
  a.dv = dv; a.sc = sc; a.e0 = e0; a.units = U;
  a.sigma_L = io.sigma_L; a.sigma_R = io.sigma_R; a.fL = a.fR = nullptr;
  a.SigL = a.SigG = nullptr;
  a.i_diag = 0; a.i_off = -1; a.Adiag = D; a.Aup = a.Alow = nullptr;
  ctx->launches += 4;
  CU(assemble(a, s));                                                          // D_0 = A_00
  CU(cudaMemsetAsync(dDt, 0, blk * (size_t)U, s));
  CU(bcopy(S1(Ft), shared(Arow, 0), b, U, s));                                // F_t0 = A_t0
  CU(bcopy(S1(Fc), shared(Acol, 0), b, U, s));                                // F_0t = A_0t
  tip_assemble_kernel<<<eg, 256, 0, s>>>(S1(Att), ar.H_tip, dv.E, dv.eta, e0, b);
  CU(cudaGetLastError());
  // ---------------- elimination of every device block, the tip kept
  for (int k = 0; k < nb; ++k) {
    CU(eng.inverse(outD(k), S1(D), b, U, st, S1(T1), S1(T2)));                 // g_k (in the G_kk output)
    CU(eng.gemm(fac(Xtf, k), S1(Ft), OP_N, outD(k), OP_N, ONE, NOMAT, ZERO, b, U));     // Xt_k = F_tk g_k
    CU(eng.gemm(fac(Wtf, k), outD(k), OP_N, S1(Fc), OP_N, ONE, NOMAT, ZERO, b, U));     // Wt_k = g_k F_kt
    CU(eng.gemm(S1(dDt), fac(Xtf, k), OP_N, S1(Fc), OP_N, MONE, S1(dDt), ONE, b, U));   // dD_t -= Xt_k F_kt
    if (k + 1 == nb) break;
    a.i_diag = k + 1; a.i_off = k;
    a.Adiag = Adiag; a.Aup = Aup; a.Alow = Alow;
    ++ctx->launches;
    CU(assemble(a, s));                                                        // A_jj, A_kj, A_jk
    CU(eng.gemm(fac(Yf, k), S1(Alow), OP_N, outD(k), OP_N, ONE, NOMAT, ZERO, b, U));    // Y_k = A_jk g_k
    CU(eng.gemm(fac(Xf, k), outD(k), OP_N, S1(Aup), OP_N, ONE, NOMAT, ZERO, b, U));     // X_k = g_k A_kj
    CU(eng.gemm(S1(D), fac(Yf, k), OP_N, S1(Aup), OP_N, MONE, S1(Adiag), ONE, b, U));   // D_j
    CU(eng.gemm(S1(Ft2), fac(Xtf, k), OP_N, S1(Aup), OP_N, MONE, shared(Arow, k + 1), ONE, b, U));   // F_tj
    CU(eng.gemm(S1(Fc2), fac(Yf, k), OP_N, S1(Fc), OP_N, MONE, shared(Acol, k + 1), ONE, b, U));    // F_jt
    std::swap(Ft, Ft2);
    std::swap(Fc, Fc2);
  }
  // ---------------- the tip: G_tt = (A_tt + dD_t)^{-1}
  ++ctx->launches;
  add_kernel<<<eg, 256, 0, s>>>(S1(T0), S1(Att), S1(dDt), b, nullptr);
  CU(cudaGetLastError());
  CU(eng.inverse(Gtt, S1(T0), b, U, st, S1(T1), S1(T2)));
  // ---------------- reconstruction from the last block up
  for (int k = nb - 1; k >= 0; --k) {
    const bool last = k + 1 == nb;
    // G_tk = -(G_tt Xt_k) [- G_tj Y_k]
    if (last) {
      CU(eng.gemm(arr(ar.Grow, k), Gtt, OP_N, fac(Xtf, k), OP_N, MONE, NOMAT, ZERO, b, U));
      CU(eng.gemm(arr(ar.Gcol, k), fac(Wtf, k), OP_N, Gtt, OP_N, MONE, NOMAT, ZERO, b, U));
      // G_kk = g_k - Wt_k G_tk
      CU(eng.gemm(outD(k), fac(Wtf, k), OP_N, arr(ar.Grow, k), OP_N, MONE, outD(k), ONE, b, U));
    } else {
      const BMat Gjj = outD(k + 1);
      const BMat Gtj_ = arr(ar.Grow, k + 1), Gjt_ = arr(ar.Gcol, k + 1);
      CU(eng.gemm(S1(T0), Gtt, OP_N, fac(Xtf, k), OP_N, ONE, NOMAT, ZERO, b, U));
      CU(eng.gemm(arr(ar.Grow, k), Gtj_, OP_N, fac(Yf, k), OP_N, MONE, S1(T0), MONE, b, U));       // G_tk
      CU(eng.gemm(S1(T0), fac(Wtf, k), OP_N, Gtt, OP_N, ONE, NOMAT, ZERO, b, U));
      CU(eng.gemm(arr(ar.Gcol, k), fac(Xf, k), OP_N, Gjt_, OP_N, MONE, S1(T0), MONE, b, U));      // G_kt
      CU(eng.gemm(S1(T0), Gjt_, OP_N, fac(Xtf, k), OP_N, ONE, NOMAT, ZERO, b, U));
      CU(eng.gemm(offB(io.GRl, k), Gjj, OP_N, fac(Yf, k), OP_N, MONE, S1(T0), MONE, b, U));       // G_jk
      CU(eng.gemm(S1(T0), fac(Wtf, k), OP_N, Gtj_, OP_N, ONE, NOMAT, ZERO, b, U));
      CU(eng.gemm(offB(io.GRu, k), fac(Xf, k), OP_N, Gjj, OP_N, MONE, S1(T0), MONE, b, U));       // G_kj
      // G_kk = g_k - Wt_k G_tk - X_k G_jk
      CU(eng.gemm(outD(k), fac(Wtf, k), OP_N, arr(ar.Grow, k), OP_N, MONE, outD(k), ONE, b, U));
      CU(eng.gemm(outD(k), fac(Xf, k), OP_N, offB(io.GRl, k), OP_N, MONE, outD(k), ONE, b, U));
    }
  }
  return NEGF_OK;
}

size_t rgf_bytes_per_energy(int nb, int b, const RgfIO& io, int mixed) {
  const size_t blk = sizeof(zc) * (size_t)b * b;
  const bool greater = io.lesser && io.greater;
  size_t n = 3 + (io.lesser ? 1 : 0) + (greater ? 1 : 0) + 4 + std::max(nb - 1, 1);
  if (rgf_small_supported(b, mixed))   // blocks assembled for every index (one launch)
    n += (size_t)(nb - 1) * (1 + (io.lesser ? 1 : 0) + (greater ? 1 : 0)) + 2 * (size_t)(std::max(nb - 1, 1) - 1);
  if (!io.GRd) n += nb;
  if (io.lesser && !io.GLd) n += nb;
  if (greater && !io.GGd) n += nb;
  if (!io.GRu) n += 1;
  size_t bytes = n * blk;
  bytes += zinv_scratch_bytes(b, 1, mixed ? 1 : 0);
  // the sliced products' scratch, and a second one for the 5-digit correction products
  if (mixed == 1) bytes += 2 * (ozt_scratch_bytes(b, 1) + 1024);
  return bytes;
}

// ---------------------------------------------------------------------------
// OBC: decimation + Newton polishing, FP64, units = (side, energy)
// ---------------------------------------------------------------------------
struct LeadArgs {
  DevView dv;
  int e0, U;
  zc *a00, *al0, *be0, *eps, *epss, *al, *be;   // slot bases, unit stride b*b, 2U units
  // units of a batched group: energy unit_e[k] of device udev[unit_dev[k]] (then dv and
  // e0 are unused)
  const UnitDev* udev = nullptr;
  const int* unit_dev = nullptr;
  const int* unit_e = nullptr;
};

// unit u < U: left lead of energy e0+u; u >= U: right lead of energy e0+u-U
__global__ void lead_init_kernel(LeadArgs a) {
  const int u = blockIdx.y;
  const bool left = u < a.U;
  const int k = left ? u : u - a.U;   // the energy unit
  int e = a.e0 + k;
  if (a.udev) {
    a.dv = a.udev[a.unit_dev[k]].dv;
    e = a.unit_e[k];
  }
  const int b = a.dv.b, nb = a.dv.nb;
  const long long bb = (long long)b * b;
  const zc z = zmake(a.dv.E[e], a.dv.eta);
  const int cd = left ? 0 : nb - 1;   // lead cell copies this device block
  const int cu = left ? 0 : nb - 2;   // ... and this hop
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < bb;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / b), c = (int)(idx - (long long)r * b);
    const long long cr = (long long)c * b + r;
    zc s00 = a.dv.Sd ? a.dv.Sd[cd * bb + idx] : zmake(r == c ? 1.0 : 0.0, 0.0);
    zc a00 = zsub(zmul(z, s00), a.dv.Hd[cd * bb + idx]);
    zc s01 = a.dv.Su ? a.dv.Su[cu * bb + idx] : zmake(0.0, 0.0);
    zc a01 = zsub(zmul(z, s01), a.dv.Hu[cu * bb + idx]);
    zc s10 = a.dv.Su ? zconj(a.dv.Su[cu * bb + cr]) : zmake(0.0, 0.0);
    zc a10 = zsub(zmul(z, s10), zconj(a.dv.Hu[cu * bb + cr]));
    // right lead: alpha = a01 (towards the lead interior), beta = a10; left lead: swapped
    const zc al = left ? a10 : a01;
    const zc be = left ? a01 : a10;
    const long long o = u * bb + idx;
    a.a00[o] = a00; a.eps[o] = a00; a.epss[o] = a00;
    a.al0[o] = al; a.al[o] = al;
    a.be0[o] = be; a.be[o] = be;
  }
}

// per unit: m = max(max|al|, max|be|).  mode 0: ref[u] = m.  mode 1: convergence check.
__global__ void lead_norm_kernel(BMat al, BMat be, int n, int mode, double* ref, int* done, int* live, int* iters,
                                 int it, double tol, int* n_active, const int* skip = nullptr) {
  const int u = blockIdx.x;
  if (mode == 1 && done[u]) return;
  if (mode == 0 && skip && skip[u]) {   // solved by the warm start: no decimation
    if (threadIdx.x == 0) {
      ref[u] = 1.0;
      done[u] = 1;
      live[u] = 0;
      iters[u] = 0;
    }
    return;
  }
  const long long nn = (long long)n * n;
  const zc* x = al.at(u);
  const zc* y = be.at(u);
  // the largest |entry|, from the squared moduli (two FP64 operations per entry; one
  // square root per block)
  double m = 0.0;
  for (long long i = threadIdx.x; i < nn; i += blockDim.x) {
    m = fmax(m, zabs2(x[i]));
    m = fmax(m, zabs2(y[i]));
  }
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    m = sqrt(m);
    if (mode == 0) {
      ref[u] = fmax(m, 1e-300);
      done[u] = 0;
      live[u] = 1;
      iters[u] = 0;
    } else {
      if (m < tol * ref[u] || !isfinite(m)) {
        done[u] = isfinite(m) ? 1 : 2;
        live[u] = 0;
        iters[u] = it;
      } else if (n_active) {
        atomicAdd(n_active, 1);
      }
    }
  }
}

// eps_s -= agb; eps -= agb + bga
__global__ void lead_update_kernel(BMat eps, BMat epss, BMat agb, BMat bga, int n, const int* done) {
  const int u = blockIdx.y;
  if (done[u]) return;
  const long long nn = (long long)n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x) {
    const zc x = agb.at(u)[i];
    epss.at(u)[i] = zsub(epss.at(u)[i], x);
    eps.at(u)[i] = zsub(zsub(eps.at(u)[i], x), bga.at(u)[i]);
  }
}

// F = KG - I (in place), res[u] = ||F||_F / sqrt(n); mode 1 stores into resn instead
__global__ void residual_kernel(BMat F, int n, double* res, const int* active) {
  const int u = blockIdx.x;
  if (active && !active[u]) return;
  const long long nn = (long long)n * n;
  zc* f = F.at(u);
  double s = 0.0;
  for (long long i = threadIdx.x; i < nn; i += blockDim.x) {
    const int r = (int)(i / n), c = (int)(i - (long long)r * n);
    zc v = f[i];
    if (r == c) v.x -= 1.0;
    f[i] = v;
    s += v.x * v.x + v.y * v.y;
  }
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    res[u] = sqrt(s / n);
  }
}

// redo[u] = 1 for an active unit whose refined inverse is not FP64-class: the residual
// R = I - M X left by the last refinement step (the step from X to X + X R leaves an
// error of the order of |R|^2) has a Frobenius norm above tol, or is not finite
__global__ void refine_check_kernel(BMat R, int n, const int* active, double tol, int* redo) {
  const int u = blockIdx.x;
  if (active && !active[u]) {
    if (threadIdx.x == 0) redo[u] = 0;
    return;
  }
  const zc* r = R.at(u);
  const int nn = n * n;
  double s = 0.0;
  for (int i = threadIdx.x; i < nn; i += blockDim.x) s += r[i].x * r[i].x + r[i].y * r[i].y;
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    redo[u] = (s <= tol * tol) ? 0 : 1;   // NaN: redo
  }
}

// Smith step bookkeeping: S += inc; conv if max|inc| <= tol max|S|; rebalance P, Q
__global__ void smith_accum_kernel(BMat S, BMat inc, int n, int* act, double tol) {
  const int u = blockIdx.x;
  if (!act[u]) return;
  const long long nn = (long long)n * n;
  zc* s = S.at(u);
  const zc* d = inc.at(u);
  double mi = 0.0, ms = 0.0;   // squared moduli
  for (long long i = threadIdx.x; i < nn; i += blockDim.x) {
    zc v = zadd(s[i], d[i]);
    s[i] = v;
    mi = fmax(mi, zabs2(d[i]));
    ms = fmax(ms, zabs2(v));
  }
  __shared__ double r1[32], r2[32];
  for (int off = 16; off > 0; off >>= 1) {
    mi = fmax(mi, __shfl_down_sync(0xffffffffu, mi, off));
    ms = fmax(ms, __shfl_down_sync(0xffffffffu, ms, off));
  }
  if ((threadIdx.x & 31) == 0) { r1[threadIdx.x >> 5] = mi; r2[threadIdx.x >> 5] = ms; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { mi = fmax(mi, r1[w]); ms = fmax(ms, r2[w]); }
    mi = sqrt(mi);
    ms = sqrt(ms);
    if (mi <= tol * fmax(ms, 1e-300) || !isfinite(ms)) act[u] = 0;
  }
}

__global__ void balance_kernel(BMat P, BMat Q, int n, const int* act) {
  const int u = blockIdx.x;
  if (!act[u]) return;
  const long long nn = (long long)n * n;
  zc* p = P.at(u);
  zc* q = Q.at(u);
  double mp = 0.0, mq = 0.0;   // squared moduli
  for (long long i = threadIdx.x; i < nn; i += blockDim.x) {
    mp = fmax(mp, zabs2(p[i]));
    mq = fmax(mq, zabs2(q[i]));
  }
  __shared__ double r1[32], r2[32];
  __shared__ double sc;
  for (int off = 16; off > 0; off >>= 1) {
    mp = fmax(mp, __shfl_down_sync(0xffffffffu, mp, off));
    mq = fmax(mq, __shfl_down_sync(0xffffffffu, mq, off));
  }
  if ((threadIdx.x & 31) == 0) { r1[threadIdx.x >> 5] = mp; r2[threadIdx.x >> 5] = mq; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { mp = fmax(mp, r1[w]); mq = fmax(mq, r2[w]); }
    sc = (mp > 0.0 && mq > 0.0) ? sqrt(sqrt(mq) / sqrt(mp)) : 1.0;
  }
  __syncthreads();
  const double s = sc;
  for (long long i = threadIdx.x; i < nn; i += blockDim.x) {
    p[i] = zscale(p[i], s);
    q[i] = zscale(q[i], 1.0 / s);
  }
}

// Newton acceptance: if resn < res: g = gn, res = resn
__global__ void newton_accept_kernel(BMat g, BMat gn, int n, double* res, const double* resn, int* need,
                                     double target, int* steps) {
  const int u = blockIdx.x;
  if (!need[u]) return;
  const bool take = resn[u] < res[u];
  if (take) {
    const long long nn = (long long)n * n;
    for (long long i = threadIdx.x; i < nn; i += blockDim.x) g.at(u)[i] = gn.at(u)[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (take) res[u] = resn[u];
    need[u] = (take && res[u] > target) ? 1 : 0;
    ++steps[u];
  }
}

// warm-start Newton: every finite step is taken; a non-finite one ends the unit's
// attempt (res = inf, so that the retarded-root test rejects it)
__global__ void newton_take_kernel(BMat g, BMat gn, int n, double* res, const double* resn, int* need,
                                   double target, int* steps) {
  const int u = blockIdx.x;
  if (!need[u]) return;
  const bool fin = isfinite(resn[u]);
  if (fin) {
    const long long nn = (long long)n * n;
    for (long long i = threadIdx.x; i < nn; i += blockDim.x) g.at(u)[i] = gn.at(u)[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    ++steps[u];
    if (fin) {
      res[u] = resn[u];
      need[u] = res[u] > target ? 1 : 0;
    } else {
      res[u] = INFINITY;
      need[u] = 0;
    }
  }
}

// g[u] = the guess of its side (left units u < U, right units u >= U), warm[u] = 1 when given
__global__ void guess_init_kernel(BMat g, const zc* g0L, const zc* g0R, int U, int n, int* warm,
                                  const long long* off = nullptr) {
  const int u = blockIdx.y;
  const bool left = u < U;
  const zc* src = left ? g0L : g0R;
  if (blockIdx.x == 0 && threadIdx.x == 0) warm[u] = src ? 1 : 0;
  if (!src) return;
  const long long nn = (long long)n * n;
  const int k = left ? u : u - U;
  src += off ? off[k] : (long long)k * nn;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x)
    g.at(u)[i] = src[i];
}

__global__ void need_warm_kernel(const int* warm, const double* res, int* need, int units, double target) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < units) need[u] = (warm[u] && res[u] > target) ? 1 : 0;
}

// retarded-root test of the warm result: keep[u] = 1 when the unit had a guess, its
// residual is <= accept, and every LDL^H pivot (no pivoting) of A = i (g - g^H) exceeds
// -tol * max_k A_kk (a pivot within +-tol of zero is a semidefinite direction and is
// skipped).  A is factorised in place in the scratch block W.
__global__ void retarded_check_kernel(BMat g, BMat W, int n, const int* warm, const double* res, double accept,
                                      double tol, int* keep) {
  const int u = blockIdx.x;
  if (!warm[u] || !(res[u] <= accept)) {
    if (threadIdx.x == 0) keep[u] = 0;
    return;
  }
  const long long nn = (long long)n * n;
  const zc* x = g.at(u);
  zc* A = W.at(u);
  double mx = 0.0;
  for (long long idx = threadIdx.x; idx < nn; idx += blockDim.x) {
    const int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
    const zc a = x[idx], c = x[(long long)j * n + i];
    // A_ij = i (g_ij - conj(g_ji))
    A[idx] = zmake(-(a.y + c.y), a.x - c.x);
    if (i == j) mx = fmax(mx, -2.0 * a.y);
  }
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) mx = fmax(mx, __shfl_down_sync(0xffffffffu, mx, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  __shared__ double s_scale;
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) mx = fmax(mx, red[w]);
    s_scale = fmax(mx, 1e-300);
  }
  for (int k = 0; k < n; ++k) {
    __syncthreads();
    const double d = A[(long long)k * n + k].x;
    if (d < -tol * s_scale || !isfinite(d)) {
      if (threadIdx.x == 0) keep[u] = 0;
      return;
    }
    if (d <= tol * s_scale) continue;
    const int m = n - k - 1;
    const double inv = 1.0 / d;
    for (long long idx = threadIdx.x; idx < (long long)m * m; idx += blockDim.x) {
      const int i = k + 1 + (int)(idx / m), j = k + 1 + (int)(idx % m);
      const zc l = A[(long long)i * n + k], r = A[(long long)k * n + j];
      zc& t = A[(long long)i * n + j];
      t.x -= (l.x * r.x - l.y * r.y) * inv;
      t.y -= (l.x * r.y + l.y * r.x) * inv;
    }
  }
  if (threadIdx.x == 0) keep[u] = 1;
}

__global__ void not_kernel(const int* a, int* out, int units) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < units) out[u] = a[u] ? 0 : 1;
}

// off[0 .. c-1] = u * bb for the c units with mask[u] != 0, in increasing u (one CTA
// of 1024 threads: ballots within warps, a scan of the warp counts per tile of 1024)
__global__ void __launch_bounds__(1024) compact_kernel(const int* mask, int units, long long bb, long long* off) {
  __shared__ int wsum[32];
  __shared__ int s_base;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) s_base = 0;
  __syncthreads();
  for (int i0 = 0; i0 < units; i0 += 1024) {
    const int i = i0 + tid;
    const int f = (i < units && mask[i]) ? 1 : 0;
    const unsigned bal = __ballot_sync(0xffffffffu, f);
    const int pre = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    if (w == 0) {   // exclusive prefix of the 32 warp counts
      const int v = wsum[lane];
      int x = v;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      wsum[lane] = x - v;
    }
    __syncthreads();
    const int base = s_base;
    if (f) off[base + wsum[w] + pre] = (long long)i * bb;
    __syncthreads();
    if (tid == 1023) s_base = base + wsum[31] + __popc(bal);
    __syncthreads();
  }
}

__global__ void count_kernel(const int* flags, int units, int* out) {
  int c = 0;
  for (int u = threadIdx.x; u < units; u += blockDim.x) c += flags[u] != 0;
  for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(0xffffffffu, c, off);
  __shared__ int red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) c += red[w];
    *out = c;
  }
}

__global__ void set_need_kernel(const double* res, int* need, int units, double target, const int* only) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < units) need[u] = (only[u] && res[u] > target) ? 1 : 0;
}

__global__ void obc_finish_kernel(const int* done, const double* res, const int* iters, const int* nsteps, int U,
                                  int32_t* status, int32_t* iters_out, int32_t* newton_out, double accept,
                                  const int* glob = nullptr) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= U) return;
  const int ge = glob ? glob[e] : e;   // the energy's index in the outputs
  const bool okL = done[e] == 1 && res[e] <= accept;
  const bool okR = done[U + e] == 1 && res[U + e] <= accept;
  if (status) status[ge] = (okL && okR) ? NEGF_OK : NEGF_ERR_NOCONV;
  if (iters_out) {
    iters_out[2 * ge] = iters[e];
    iters_out[2 * ge + 1] = iters[U + e];
  }
  if (newton_out) {
    newton_out[2 * ge] = nsteps[e];
    newton_out[2 * ge + 1] = nsteps[U + e];
  }
}

// ---------------------------------------------------------------------------
// observables (row a9), FP64 with fixed-order tree reductions
// ---------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < NT / 32; ++w) t += red[w];
  __syncthreads();
  return t;   // valid in thread 0
}

// Gamma = i (Sigma - Sigma^H)
__global__ void gamma_kernel(BMat G, BMat Sg, int n) {
  const int u = blockIdx.y;
  const long long nn = (long long)n * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn; i += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(i / n), c = (int)(i - (long long)r * n);
    const zc d = zsub(Sg.at(u)[i], zconj(Sg.at(u)[(long long)c * n + r]));
    G.at(u)[i] = zmake(-d.y, d.x);
  }
}

// T = Re( Tr[Gam i (G - G^H)] - sum_pq K1_pq conj(K2_pq) ),  K1 = Gam G, K2 = G Gam
__global__ void transmission_kernel(BMat Gam, BMat G, BMat K1, BMat K2, int n, double* T) {
  const int u = blockIdx.x;
  const long long nn = (long long)n * n;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < nn; i += blockDim.x) {
    const int p = (int)(i / n), q = (int)(i - (long long)p * n);
    // Gam_pq * i (G_qp - conj(G_pq))
    const zc gqp = G.at(u)[(long long)q * n + p];
    const zc gpq = G.at(u)[i];
    const zc d = zsub(gqp, zconj(gpq));
    const zc id = zmake(-d.y, d.x);
    const zc gam = Gam.at(u)[i];
    acc += gam.x * id.x - gam.y * id.y;
    const zc k1 = K1.at(u)[i], k2 = K2.at(u)[i];
    acc -= k1.x * k2.x + k1.y * k2.y;   // Re(k1 conj(k2))
  }
  __shared__ double red[32];
  const double t = block_sum<256>(acc, red);
  if (threadIdx.x == 0) T[u] = t;
}

// Traces of block products by 32 x 32 tiles (256 threads, warp w takes rows w, w+8, ..,
// lane l columns c0 + l): acc[k] += Re (PART 0) or Im (PART 1) of sum_l X[r][l] Y[l][r]
// for row r = r0 + w + 8k of X, with Y read as row segments into shared memory and used
// transposed, so that both blocks are read with coalesced row segments (one part: two
// FP64 FMAs per element).  ly(l, r) gives Y[l][r] (0 <= l, r < b).
template <int PART, class LY>
__device__ __forceinline__ void tile_rowdot(const zc* __restrict__ X, LY ly, int b, int r0, zc (*sm)[33],
                                            double acc[4]) {
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int c0 = 0; c0 < b; c0 += 32) {
    __syncthreads();   // the previous tile has been used
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int l = c0 + ty + 8 * k, r = r0 + tx;
      sm[ty + 8 * k][tx] = (l < b && r < b) ? ly(l, r) : zmake(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int r = r0 + ty + 8 * k, l = c0 + tx;
      if (r < b && l < b) {
        const zc x = X[r * b + l], y = sm[tx][ty + 8 * k];
        acc[k] = PART == 0 ? fma(x.x, y.x, fma(-x.y, y.y, acc[k])) : fma(x.x, y.y, fma(x.y, y.x, acc[k]));
      }
    }
  }
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  return v;   // valid in lane 0
}

// DOS(E) = -(1/pi) Im Tr[G S] over the BT pattern: part[u][i] = Im of block row i's share
// (G_ii S_ii and, below the last block, G_{i,i+1} S_{i+1,i} + G_{i+1,i} S_{i,i+1}), one
// CTA per (block, energy); dos_sum_kernel adds the shares in block order
__global__ void __launch_bounds__(256) dos_part_kernel(DevView dv, const zc* GRd, const zc* GRu, const zc* GRl, int e0,
                                                       int eg, double* part) {
  const int i = blockIdx.x, u = blockIdx.y, eb = e0 + u - eg;   // eb: the energy's place in the G buffers
  const int nb = dv.nb, b = dv.b;
  const long long bb = (long long)b * b;
  __shared__ zc sm[32][33];
  __shared__ double red[32];
  const zc* g = GRd + ((long long)eb * nb + i) * bb;
  double acc = 0.0;
  if (!dv.Sd) {
    for (int r = threadIdx.x; r < b; r += blockDim.x) acc += g[r * b + r].y;
  } else {
    const zc* S = dv.Sd + i * bb;
    for (int r0 = 0; r0 < b; r0 += 32) {
      double t[4] = {0.0, 0.0, 0.0, 0.0};
      tile_rowdot<1>(g, [&](int l, int r) { return S[l * b + r]; }, b, r0, sm, t);
      acc += t[0] + t[1] + t[2] + t[3];
    }
  }
  if (dv.Su && GRu && GRl && i + 1 < nb) {
    const zc* gu = GRu + ((long long)eb * (nb - 1) + i) * bb;
    const zc* gl = GRl + ((long long)eb * (nb - 1) + i) * bb;
    const zc* Su = dv.Su + i * bb;
    // G_{i,i+1}[p][q] S_{i+1,i}[q][p] with S_{i+1,i} = S_up^H: elementwise with conj(Su)
    for (int k = threadIdx.x; k < b * b; k += blockDim.x) acc = fma(gu[k].y, Su[k].x, fma(-gu[k].x, Su[k].y, acc));
    // G_{i+1,i}[p][q] S_{i,i+1}[q][p]
    for (int r0 = 0; r0 < b; r0 += 32) {
      double t[4] = {0.0, 0.0, 0.0, 0.0};
      tile_rowdot<1>(gl, [&](int l, int r) { return Su[l * b + r]; }, b, r0, sm, t);
      acc += t[0] + t[1] + t[2] + t[3];
    }
  }
  const double v = block_sum<256>(acc, red);
  if (threadIdx.x == 0) part[(long long)u * nb + i] = v;
}

__global__ void dos_sum_kernel(const double* part, int nb, int e0, int U, double* dos) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= U) return;
  double t = 0.0;
  for (int i = 0; i < nb; ++i) t += part[(long long)u * nb + i];
  dos[e0 + u] = -t / M_PI;
}

// J_i(E) = 2 Re Tr[(H_{i,i+1} - z S_{i,i+1}) G^<_{i+1,i}], one CTA per (energy, interface)
__global__ void __launch_bounds__(256) current_kernel(DevView dv, const zc* GLl, int e0, int eg, double* J) {
  const int u = blockIdx.y, e = e0 + u, i = blockIdx.x;
  const int nb = dv.nb, b = dv.b;
  const long long bb = (long long)b * b;
  const zc z = zmake(dv.E[e], dv.eta);
  const zc* g = GLl + ((long long)(e - eg) * (nb - 1) + i) * bb;
  const zc* H = dv.Hu + i * bb;
  const zc* S = dv.Su ? dv.Su + i * bb : nullptr;
  __shared__ zc sm[32][33];
  __shared__ double red[32];
  // sum_qp G[q][p] A[p][q], A = H - z S (shared by all energies, read in row segments)
  double acc = 0.0;
  for (int r0 = 0; r0 < b; r0 += 32) {
    double t[4] = {0.0, 0.0, 0.0, 0.0};
    tile_rowdot<0>(g, [&](int l, int r) {
      zc x = H[l * b + r];
      if (S) x = zsub(x, zmul(z, S[l * b + r]));
      return x;
    }, b, r0, sm, t);
    acc += t[0] + t[1] + t[2] + t[3];
  }
  const double v = block_sum<256>(acc, red);
  if (threadIdx.x == 0) J[(long long)e * (nb - 1) + i] = 2.0 * v;
}

// per-energy orbital occupation Re(-i (G^< S)_kk)/(2 pi) into nE[u][k], k = i b + r over
// nb*b, one CTA per (block row i, energy)
__global__ void __launch_bounds__(256) density_energy_kernel(DevView dv, const zc* GLd, const zc* GLl, int e0, int eg,
                                                             double* nE) {
  const int i = blockIdx.x, u = blockIdx.y, e = e0 + u - eg;   // the energy's place in the G buffers
  const int nb = dv.nb, b = dv.b;
  const long long bb = (long long)b * b;
  const long long N = (long long)nb * b;
  const zc* gd = GLd + ((long long)e * nb + i) * bb;
  double* out = nE + (long long)u * N + (long long)i * b;
  if (!dv.Sd) {
    for (int r = threadIdx.x; r < b; r += blockDim.x) out[r] = gd[r * b + r].y / (2.0 * M_PI);
    return;
  }
  __shared__ zc sm[32][33];
  const zc* S = dv.Sd + i * bb;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r0 = 0; r0 < b; r0 += 32) {
    double t[4] = {0.0, 0.0, 0.0, 0.0};   // imaginary parts
    // (G^<_ii S_ii)_rr
    tile_rowdot<1>(gd, [&](int l, int r) { return S[l * b + r]; }, b, r0, sm, t);
    if (i + 1 < nb) {
      // (G^<_{i,i+1} S_{i+1,i})_rr with G^<_{i,i+1}[r][l] = -conj(G^<_{i+1,i}[l][r]) and
      // S_{i+1,i}[l][r] = conj(Su[r][l]): -conj(sum_l Su[r][l] G^<_{i+1,i}[l][r]), whose
      // imaginary part is that of the sum
      const zc* gl = GLl + ((long long)e * (nb - 1) + i) * bb;
      tile_rowdot<1>(dv.Su + i * bb, [&](int l, int r) { return gl[l * b + r]; }, b, r0, sm, t);
    }
    if (i > 0) {   // (G^<_{i,i-1} S_{i-1,i})_rr
      const zc* gl = GLl + ((long long)e * (nb - 1) + (i - 1)) * bb;
      const zc* Su = dv.Su + (i - 1) * bb;
      tile_rowdot<1>(gl, [&](int l, int r) { return Su[l * b + r]; }, b, r0, sm, t);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double m = warp_sum(t[k]);
      const int r = r0 + ty + 8 * k;
      if (tx == 0 && r < b) out[r] = m / (2.0 * M_PI);   // Re(-i m) = Im m
    }
  }
}

// density[k] += sum_u w[e0+u] nE[u][k]  (fixed order over u)
__global__ void density_accum_kernel(const double* nE, const double* w, int e0, int U, long long N, double* dens) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N; k += (long long)gridDim.x * blockDim.x) {
    double acc = dens[k];
    for (int u = 0; u < U; ++u) acc += w[e0 + u] * nE[(long long)u * N + k];
    dens[k] = acc;
  }
}

// the observables' inputs and outputs of one device (device-offset pointers); the G
// blocks may start at any energy eg of the device ([e - eg][nb] / [e - eg][nb - 1])
struct ObsIO {
  const zc* sigma_L;
  const double* w;
  const zc *GRd, *GRu, *GRl, *GLd, *GLl;
  double *T, *dos, *current, *density;
};

size_t observables_bytes_per_energy(const DevView& dv, int sl) {
  const long long bb = (long long)dv.b * dv.b, N = (long long)dv.nb * dv.b;
  return std::max<size_t>(sizeof(zc) * (size_t)bb * 4 + (sl ? ozt_scratch_bytes(dv.b, 1) + 1024 : 0),
                          sizeof(double) * (size_t)N);
}

// observables of energies e0 .. e0+U-1 (row a9), with ws as scratch; sl: T's two block
// products on the sliced tensor-core path
negf_status observables_chunk(Ctx* ctx, Engine& eng, const DevView& dv, const ObsIO& ob, int sl, int e0, int U,
                              int eg, char* ws) {
  cudaStream_t s = eng.s;
  const int b = dv.b, nb = dv.nb;
  const long long bb = (long long)b * b;
  const long long N = (long long)nb * b;
  eng.mixed = sl;
  if (ob.T) {
    zc* p = (zc*)ws;
    BMat Gam{p, bb}, K1{p + (long long)U * bb, bb}, K2{p + 2LL * U * bb, bb};
    eng.ozt_scratch = sl ? (void*)(((uintptr_t)(p + 3LL * U * bb) + 1023) & ~(uintptr_t)1023) : nullptr;
    BMat Sg{(zc*)ob.sigma_L + (long long)e0 * bb, bb};
    BMat G00{(zc*)ob.GRd + (long long)(e0 - eg) * nb * bb, (long long)nb * bb};
    dim3 grid((unsigned)std::min<long long>((bb + 255) / 256, 1024), U);
    gamma_kernel<<<grid, 256, 0, s>>>(Gam, Sg, b);
    KCHECK();
    CU(eng.gemm(K1, Gam, OP_N, G00, OP_N, ONE, NOMAT, ZERO, b, U));
    CU(eng.gemm(K2, G00, OP_N, Gam, OP_N, ONE, NOMAT, ZERO, b, U));
    transmission_kernel<<<U, 256, 0, s>>>(Gam, G00, K1, K2, b, ob.T + e0);
    KCHECK();
  }
  if (ob.dos) {
    double* part = (double*)ws;   // [U][nb] block-row shares (ws holds >= N doubles per energy)
    dos_part_kernel<<<dim3(nb, U), 256, 0, s>>>(dv, ob.GRd, ob.GRu, ob.GRl, e0, eg, part);
    KCHECK();
    dos_sum_kernel<<<(U + 255) / 256, 256, 0, s>>>(part, nb, e0, U, ob.dos);
    KCHECK();
  }
  if (ob.current && nb > 1) {
    current_kernel<<<dim3(nb - 1, U), 256, 0, s>>>(dv, ob.GLl, e0, eg, ob.current);
    KCHECK();
  }
  if (ob.density) {
    double* nE = (double*)ws;
    density_energy_kernel<<<dim3(nb, U), 256, 0, s>>>(dv, ob.GLd, ob.GLl, e0, eg, nE);
    KCHECK();
    density_accum_kernel<<<(unsigned)std::min<long long>((N + 255) / 256, 1024), 256, 0, s>>>(nE, ob.w, e0, U, N,
                                                                                                ob.density);
    KCHECK();
  }
  return NEGF_OK;
}

}  // namespace

void negf::negf_set_error_message(const char* msg) { g_tls_error = msg ? msg : ""; }

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

negf_status negf_ctx_create(negf_ctx** out, int device, size_t workspace_bytes) {
  Ctx* ctx = nullptr;
  if (!out) return fail(nullptr, NEGF_ERR_ARG, "out pointer is NULL");
  *out = nullptr;
  ctx = new Ctx();
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) {
    std::string m = std::string("cudaSetDevice: ") + cudaGetErrorString(e);
    delete ctx;
    return fail(nullptr, NEGF_ERR_CUDA, m);
  }
  ctx->device = device;
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (workspace_bytes == 0) workspace_bytes = (size_t)1 << 30;
  e = cudaMalloc(&ctx->ws, workspace_bytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_err, 64);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, 64);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->h_pinned, 64);
  if (e != cudaSuccess) {
    std::string m = std::string("workspace allocation: ") + cudaGetErrorString(e);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->d_err) cudaFree(ctx->d_err);
    delete ctx;
    return fail(nullptr, NEGF_ERR_NOMEM, m);
  }
  ctx->ws_bytes = workspace_bytes;
  *out = reinterpret_cast<negf_ctx*>(ctx);
  return NEGF_OK;
}

negf_status negf_ctx_destroy(negf_ctx* c) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return NEGF_OK;
  cudaSetDevice(ctx->device);
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  for (const ProfRec& r : ctx->recs) { cudaEventDestroy(r.ev0); cudaEventDestroy(r.ev1); }
  for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
  delete ctx;
  return NEGF_OK;
}

const char* negf_last_error(const negf_ctx* c) {
  const Ctx* ctx = reinterpret_cast<const Ctx*>(c);
  if (ctx) return ctx->last_error.c_str();
  return g_tls_error.c_str();
}

negf_status negf_ctx_sync(negf_ctx* c, negf_stream stream) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaMemcpyAsync(ctx->h_pinned, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CU(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s));
  CU(cudaStreamSynchronize(s));
  const int w = ctx->h_pinned[0];
  if (w != 0) return fail(ctx, (negf_status)(-w), "device code reported status " + std::to_string(-w));
  return NEGF_OK;
}

negf_status negf_worklist(const negf_system* sys, int32_t bs, int32_t* count, int32_t* unit_dev, int32_t* unit_e,
                          int64_t* off_d, int64_t* off_o) {
  if (!count) return fail(nullptr, NEGF_ERR_ARG, "count is NULL");
  Layout L;
  negf_status st = make_layout(nullptr, sys, L);
  if (st != NEGF_OK) return st;
  std::vector<int> devs;
  for (int d = 0; d < sys->ndev; ++d)
    if (sys->ne[d] > 0 && sys->bs[d] == bs) devs.push_back(d);
  const WorkList w = make_worklist(sys, L, devs, (long long)bs * bs);
  *count = (int32_t)w.unit_dev.size();
  for (size_t u = 0; u < w.unit_dev.size(); ++u) {
    if (unit_dev) unit_dev[u] = devs[w.unit_dev[u]];
    if (unit_e) unit_e[u] = w.unit_e[u];
    if (off_d) off_d[u] = w.off_d[u];
    if (off_o) off_o[u] = w.off_o[u];
  }
  return NEGF_OK;
}

negf_status negf_layout(const negf_system* sys, int64_t* out) {
  if (!out) return fail(nullptr, NEGF_ERR_ARG, "out is NULL");
  Layout L;
  negf_status st = make_layout(nullptr, sys, L);
  if (st != NEGF_OK) return st;
  for (size_t k = 0; k < L.off.size(); ++k) out[k] = L.off[k];
  return NEGF_OK;
}

// status[glob[u]] = st_units[u]
__global__ void status_scatter_kernel(int32_t* status, const int32_t* st_units, const int* glob, int U) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u < U) status[glob[u]] = st_units[u];
}

// batched sweeps over every (device, energy) unit of the devices `devs`, which share a
// block size; units are chunked to the workspace, each chunk's tables copied ahead of
// the sweep workspace
negf_status rgf_batched_group(Ctx* ctx, Engine& eng, const negf_system* sys, const Layout& L,
                              const std::vector<int>& devs, const void* sigma_L, const void* sigma_R,
                              const double* f_L, const double* f_R, const negf_scattering* scat, void* GR_diag,
                              void* GR_up, void* GR_low, void* GL_diag, void* GL_low, void* GG_diag, void* GG_low,
                              int32_t* status, cudaStream_t s, bool lesser) {
  const int b = sys->bs[devs[0]];
  const long long bb = (long long)b * b;
  std::vector<UnitDev> ud(devs.size());
  for (size_t k = 0; k < devs.size(); ++k) {
    const int d = devs[k];
    const long long* o = &L.off[8 * (size_t)d];
    ud[k].dv = dev_view(sys, L, d);
    ud[k].sc = scat_view(scat, L, d, ud[k].dv.nb, b);
    ud[k].sigma_L = (const zc*)sigma_L + o[3];
    ud[k].sigma_R = (const zc*)sigma_R + o[3];
    ud[k].fL = f_L ? f_L + o[2] : nullptr;
    ud[k].fR = f_R ? f_R + o[2] : nullptr;
  }
  const WorkList w = make_worklist(sys, L, devs, bb);
  const int units = (int)w.unit_dev.size();
  int max_nb = 1;
  for (int d : devs) max_nb = std::max(max_nb, (int)sys->nb[d]);
  RgfIO io;
  io.sigma_L = io.sigma_R = nullptr;
  io.fL = io.fR = nullptr;
  io.GRd = (zc*)GR_diag;
  io.GRu = (zc*)GR_up;
  io.GRl = (zc*)GR_low;
  io.GLd = lesser ? (zc*)GL_diag : nullptr;
  io.GLl = lesser ? (zc*)GL_low : nullptr;
  io.GGd = lesser ? (zc*)GG_diag : nullptr;
  io.GGl = lesser ? (zc*)GG_low : nullptr;
  io.greater = lesser && (GG_diag || GG_low);
  io.status = nullptr;
  io.lesser = lesser;
  // per unit: the sweep workspace at the group's largest nb, the tables and two masks
  auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t per = rgf_bytes_per_energy(max_nb, b, io, eng.mixed) + 4 * sizeof(int) + 2 * sizeof(long long) +
                     sizeof(int32_t) + 2 * sizeof(int) * (size_t)max_nb;
  const size_t fixed = align(sizeof(UnitDev) * ud.size()) + 8 * 256 + 2048;
  if (ctx->ws_bytes <= fixed) return fail(ctx, NEGF_ERR_NOMEM, "workspace too small for the batch tables");
  int chunk = (int)std::min<size_t>((ctx->ws_bytes - fixed) / per, (size_t)65535);
  if (chunk < 1) return fail(ctx, NEGF_ERR_NOMEM, "workspace too small: one unit needs " + std::to_string(per) + " bytes");
  for (int u0 = 0; u0 < units; u0 += chunk) {
    const int U = std::min(chunk, units - u0);
    int nbc = 1;
    for (int u = u0; u < u0 + U; ++u) nbc = std::max(nbc, w.unit_nb[u]);
    std::vector<int> act_f((size_t)nbc * U), act_b((size_t)nbc * U);
    std::vector<double> frac_f(nbc), frac_b(nbc);
    for (int i = 0; i < nbc; ++i) {
      int nf = 0, nbk = 0;
      for (int u = 0; u < U; ++u) {
        const int nbu = w.unit_nb[u0 + u];
        nf += (act_f[(size_t)i * U + u] = (i < nbu) ? 1 : 0);
        nbk += (act_b[(size_t)i * U + u] = (i <= nbu - 2) ? 1 : 0);
      }
      frac_f[i] = (double)nf / U;
      frac_b[i] = (double)nbk / U;
    }
    char* p = (char*)ctx->ws;
    auto put = [&](const void* src, size_t bytes) -> void* {
      void* dst = p;
      p += align(bytes);
      return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess ? dst : nullptr;
    };
    BatchPlan bp;
    bp.nb = nbc;
    bp.udev = (const UnitDev*)put(ud.data(), sizeof(UnitDev) * ud.size());
    bp.unit_dev = (const int*)put(w.unit_dev.data() + u0, sizeof(int) * U);
    bp.unit_e = (const int*)put(w.unit_e.data() + u0, sizeof(int) * U);
    bp.off_d = (const long long*)put(w.off_d.data() + u0, sizeof(long long) * U);
    bp.off_o = (const long long*)put(w.off_o.data() + u0, sizeof(long long) * U);
    bp.act_f = (const int*)put(act_f.data(), sizeof(int) * act_f.size());
    bp.act_b = (const int*)put(act_b.data(), sizeof(int) * act_b.size());
    const int* glob = (const int*)put(w.unit_glob.data() + u0, sizeof(int) * U);
    bp.frac_f = frac_f.data();
    bp.frac_b = frac_b.data();
    bp.st_units = (int32_t*)p;
    p += align(sizeof(int32_t) * U);
    if (!bp.udev || !bp.unit_dev || !bp.unit_e || !bp.off_d || !bp.off_o || !bp.act_f || !bp.act_b || !glob)
      return fail(ctx, NEGF_ERR_CUDA, "copying the batch tables failed");
    CU(cudaMemsetAsync(bp.st_units, 0, sizeof(int32_t) * U, s));
    p = (char*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
    eng.inv_scratch = nullptr;
    negf_status st = rgf_chunk(ctx, eng, ud[0].dv, ud[0].sc, io, 0, U, p, &bp);
    if (st != NEGF_OK) return st;
    if (status) {
      ++ctx->launches;
      status_scatter_kernel<<<(U + 127) / 128, 128, 0, s>>>(status, bp.st_units, glob, U);
      CU(cudaGetLastError());
    }
  }
  return NEGF_OK;
}

static negf_status rgf_common(Ctx* ctx, const negf_system* sys, negf_precision prec, const void* sigma_L,
                              const void* sigma_R, const double* f_L, const double* f_R,
                              const negf_scattering* scat, void* GR_diag, void* GR_up, void* GR_low,
                              void* GL_diag, void* GL_low, int32_t* status, cudaStream_t s, bool lesser,
                              void* GG_diag = nullptr, void* GG_low = nullptr) {
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  Layout L;
  negf_status st = make_layout(ctx, sys, L);
  if (st != NEGF_OK) return st;
  if ((st = check_system(ctx, sys)) != NEGF_OK) return st;
  if (prec != NEGF_FP64 && prec != NEGF_MIXED && prec != NEGF_MIXED_TF32)
    return fail(ctx, NEGF_ERR_ARG, "unknown precision");
  if (!sigma_L || !sigma_R) return fail(ctx, NEGF_ERR_ARG, "sigma_L and sigma_R are required");
  if (lesser && (!f_L || !f_R)) return fail(ctx, NEGF_ERR_ARG, "f_L and f_R are required for G^<");
  if (scat && scat->per_energy != 0 && scat->per_energy != 1)
    return fail(ctx, NEGF_ERR_ARG, "scattering per_energy must be 0 or 1");
  CU(cudaSetDevice(ctx->device));
  if (status) CU(cudaMemsetAsync(status, 0, sizeof(int32_t) * L.off[8 * (size_t)sys->ndev + 2], s));
  Engine eng{ctx, s, (int)prec, nullptr};
  // devices that share a block size sweep together: one launch per step over all their
  // (device, energy) units; a device alone in its block size keeps the plain layout
  std::vector<int> sizes;
  for (int d = 0; d < sys->ndev; ++d)
    if (sys->ne[d] > 0 && std::find(sizes.begin(), sizes.end(), sys->bs[d]) == sizes.end()) sizes.push_back(sys->bs[d]);
  std::vector<char> batched(sys->ndev, 0);
  for (int bsz : sizes) {
    std::vector<int> devs;
    for (int d = 0; d < sys->ndev; ++d)
      if (sys->ne[d] > 0 && sys->bs[d] == bsz) devs.push_back(d);
    if (devs.size() < 2) continue;
    st = rgf_batched_group(ctx, eng, sys, L, devs, sigma_L, sigma_R, f_L, f_R, scat, GR_diag, GR_up, GR_low, GL_diag,
                           GL_low, GG_diag, GG_low, status, s, lesser);
    if (st != NEGF_OK) return st;
    for (int d : devs) batched[d] = 1;
  }
  for (int d = 0; d < sys->ndev; ++d) {
    const int ne = sys->ne[d];
    if (ne == 0 || batched[d]) continue;
    const DevView dv = dev_view(sys, L, d);
    const ScatView sc = scat_view(scat, L, d, dv.nb, dv.b);
    const long long* o = &L.off[8 * (size_t)d];
    RgfIO io;
    io.sigma_L = (const zc*)sigma_L + o[3];
    io.sigma_R = (const zc*)sigma_R + o[3];
    io.fL = f_L ? f_L + o[2] : nullptr;
    io.fR = f_R ? f_R + o[2] : nullptr;
    io.GRd = GR_diag ? (zc*)GR_diag + o[4] : nullptr;
    io.GRu = GR_up ? (zc*)GR_up + o[5] : nullptr;
    io.GRl = GR_low ? (zc*)GR_low + o[5] : nullptr;
    io.GLd = (lesser && GL_diag) ? (zc*)GL_diag + o[4] : nullptr;
    io.GLl = (lesser && GL_low) ? (zc*)GL_low + o[5] : nullptr;
    io.GGd = (lesser && GG_diag) ? (zc*)GG_diag + o[4] : nullptr;
    io.GGl = (lesser && GG_low) ? (zc*)GG_low + o[5] : nullptr;
    io.greater = lesser && (GG_diag || GG_low);
    io.status = status ? status + o[2] : nullptr;
    io.lesser = lesser;
    const size_t per = rgf_bytes_per_energy(dv.nb, dv.b, io, eng.mixed);
    // the device's W blocks (energy-independent part of A) ahead of the chunk workspace,
    // when there is room for them next to one energy
    const size_t wb = asm_w_bytes(dv.nb, dv.b);
    const bool use_w = ctx->ws_bytes >= wb + per;
    char* ws = (char*)ctx->ws + (use_w ? wb : 0);
    int chunk = (int)std::min<size_t>((ctx->ws_bytes - (use_w ? wb : 0)) / per, (size_t)65535);
    if (chunk < 1)
      return fail(ctx, NEGF_ERR_NOMEM, "workspace too small: one energy of this device needs " +
                                           std::to_string(per) + " bytes");
    chunk = std::min(chunk, ne);
    if (use_w) {
      zc* W = (zc*)ctx->ws;
      const long long bb = (long long)dv.b * dv.b;
      ++ctx->launches;
      asm_w_kernel<<<dim3((unsigned)std::min<long long>((bb + 255) / 256, 1024), dv.nb), 256, 0, s>>>(
          dv, W, W + dv.nb * bb, W + (2LL * dv.nb - 1) * bb);
      CU(cudaGetLastError());
      io.W = W;
    }
    for (int e0 = 0; e0 < ne; e0 += chunk) {
      const int U = std::min(chunk, ne - e0);
      eng.inv_scratch = nullptr;
      st = rgf_chunk(ctx, eng, dv, sc, io, e0, U, ws);
      if (st != NEGF_OK) return st;
    }
  }
  return NEGF_OK;
}

negf_status negf_rgf_retarded(negf_ctx* c, const negf_system* sys, negf_precision prec, const void* sigma_L,
                              const void* sigma_R, const negf_scattering* scat, void* GR_diag, void* GR_up,
                              void* GR_low, int32_t* status, negf_stream stream) {
  return rgf_common(reinterpret_cast<Ctx*>(c), sys, prec, sigma_L, sigma_R, nullptr, nullptr, scat, GR_diag,
                    GR_up, GR_low, nullptr, nullptr, status, (cudaStream_t)stream, false);
}

negf_status negf_rgf_lesser(negf_ctx* c, const negf_system* sys, negf_precision prec, const void* sigma_L,
                            const void* sigma_R, const double* f_L, const double* f_R,
                            const negf_scattering* scat, void* GR_diag, void* GR_up, void* GR_low, void* GL_diag,
                            void* GL_low, int32_t* status, negf_stream stream) {
  return rgf_common(reinterpret_cast<Ctx*>(c), sys, prec, sigma_L, sigma_R, f_L, f_R, scat, GR_diag, GR_up,
                    GR_low, GL_diag, GL_low, status, (cudaStream_t)stream, true);
}

negf_status negf_rgf_partitioned(negf_ctx* c, const negf_system* sys, negf_precision prec, int32_t P,
                                 const void* sigma_L, const void* sigma_R, const negf_scattering* scat,
                                 void* GR_diag, void* GR_up, void* GR_low, int32_t* status, negf_stream stream) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  Layout Lay;
  negf_status st = make_layout(ctx, sys, Lay);
  if (st != NEGF_OK) return st;
  if ((st = check_system(ctx, sys)) != NEGF_OK) return st;
  if (prec != NEGF_FP64 && prec != NEGF_MIXED && prec != NEGF_MIXED_TF32)
    return fail(ctx, NEGF_ERR_ARG, "unknown precision");
  if (P < 1) return fail(ctx, NEGF_ERR_ARG, "need P >= 1 partitions");
  for (int d = 0; d < sys->ndev; ++d)
    if (sys->nb[d] % P != 0 || sys->nb[d] / P < 2)
      return fail(ctx, NEGF_ERR_ARG, "device " + std::to_string(d) + ": nb must be P L with L >= 2");
  if (!sigma_L || !sigma_R) return fail(ctx, NEGF_ERR_ARG, "sigma_L and sigma_R are required");
  if (!GR_diag || !GR_up || !GR_low) return fail(ctx, NEGF_ERR_ARG, "GR_diag, GR_up and GR_low are required");
  if (scat && scat->per_energy != 0 && scat->per_energy != 1)
    return fail(ctx, NEGF_ERR_ARG, "scattering per_energy must be 0 or 1");
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaSetDevice(ctx->device));
  if (status) CU(cudaMemsetAsync(status, 0, sizeof(int32_t) * Lay.off[8 * (size_t)sys->ndev + 2], s));
  Engine eng{ctx, s, (int)prec, nullptr};
  for (int d = 0; d < sys->ndev; ++d) {
    const int ne = sys->ne[d];
    if (ne == 0) continue;
    const DevView dv = dev_view(sys, Lay, d);
    const ScatView sc = scat_view(scat, Lay, d, dv.nb, dv.b);
    const long long* o = &Lay.off[8 * (size_t)d];
    RgfIO io;
    io.sigma_L = (const zc*)sigma_L + o[3];
    io.sigma_R = (const zc*)sigma_R + o[3];
    io.fL = io.fR = nullptr;
    io.GRd = (zc*)GR_diag + o[4];
    io.GRu = (zc*)GR_up + o[5];
    io.GRl = (zc*)GR_low + o[5];
    io.GLd = io.GLl = nullptr;
    io.status = status ? status + o[2] : nullptr;
    io.lesser = false;
    const size_t per = partitioned_bytes_per_energy(dv.nb, dv.b, P, eng.mixed);
    int chunk = (int)std::min<size_t>(ctx->ws_bytes / per, (size_t)(65535 / P));
    if (chunk < 1)
      return fail(ctx, NEGF_ERR_NOMEM, "workspace too small: one energy of this device needs " +
                                           std::to_string(per) + " bytes");
    chunk = std::min(chunk, ne);
    for (int e0 = 0; e0 < ne; e0 += chunk) {
      const int U = std::min(chunk, ne - e0);
      eng.inv_scratch = nullptr;
      st = rgf_partitioned_chunk(ctx, eng, dv, sc, io, P, e0, U, (char*)ctx->ws);
      if (st != NEGF_OK) return st;
    }
  }
  return NEGF_OK;
}

negf_status negf_energy_convolution(negf_ctx* c, int32_t ne, int64_t nelem, int64_t ld, int32_t M, const double* w,
                                    const void* X, void* Y, negf_stream stream) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  if (ne < 0 || nelem < 0 || M < 0 || ld < nelem) return fail(ctx, NEGF_ERR_ARG, "need ne, nelem, M >= 0, ld >= nelem");
  if (nelem > ((int64_t)1 << 31) - 16) return fail(ctx, NEGF_ERR_ARG, "nelem beyond 2^31");
  if (!w || !X || !Y) return fail(ctx, NEGF_ERR_ARG, "NULL operand");
  if (X == Y) return fail(ctx, NEGF_ERR_ARG, "X and Y must not overlap");
  if (ne == 0 || nelem == 0) return NEGF_OK;
  if (conv_log2_size(ne, M) > 13) return fail(ctx, NEGF_ERR_ARG, "ne + M must stay <= 8192");
  const size_t need = 256 + conv_spectrum_bytes(ne, M) + sizeof(double) * (2 * (size_t)M + 1);
  if (need > ctx->ws_bytes) return fail(ctx, NEGF_ERR_NOMEM, "workspace too small for the kernel spectrum");
  CU(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  zc* Wh = (zc*)ctx->ws;
  double* wd = (double*)((char*)ctx->ws + conv_spectrum_bytes(ne, M));
  CU(cudaMemcpyAsync(wd, w, sizeof(double) * (2 * (size_t)M + 1), cudaMemcpyHostToDevice, s));
  ctx->launches += 2;
  CU(energy_convolution((const zc*)X, (zc*)Y, ld, (int)nelem, ne, M, wd, Wh, s));
  return NEGF_OK;
}

negf_status negf_scba(negf_ctx* c, const negf_system* sys, negf_precision prec, const void* sigma_L,
                      const void* sigma_R, const double* f_L, const double* f_R, const negf_boson_kernel* kern,
                      double mixing, double tol, int32_t max_iter, void* sigR_scat, void* sigL_scat,
                      void* sigG_scat, void* GR_diag, void* GR_up, void* GR_low, void* GL_diag, void* GL_low,
                      void* GG_diag, void* GG_low, int32_t* status, int32_t* iters, double* change,
                      negf_stream stream) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  Layout Lay;
  negf_status st = make_layout(ctx, sys, Lay);
  if (st != NEGF_OK) return st;
  if ((st = check_system(ctx, sys)) != NEGF_OK) return st;
  if (!kern || kern->M < 0 || !kern->w_lesser || !kern->w_greater) return fail(ctx, NEGF_ERR_ARG, "bad boson kernel");
  if (!(mixing > 0.0 && mixing <= 1.0) || !(tol > 0.0) || max_iter < 1)
    return fail(ctx, NEGF_ERR_ARG, "need 0 < mixing <= 1, tol > 0, max_iter >= 1");
  if (!sigR_scat || !sigL_scat || !sigG_scat) return fail(ctx, NEGF_ERR_ARG, "the three self-energy arrays are required");
  if (!GR_diag || !GL_diag || !GG_diag) return fail(ctx, NEGF_ERR_ARG, "GR_diag, GL_diag and GG_diag are required");
  if (!f_L || !f_R || !sigma_L || !sigma_R) return fail(ctx, NEGF_ERR_ARG, "lead self-energies and occupations required");
  const long long nel = Lay.off[8 * (size_t)sys->ndev + 4];   // diagonal-block elements, all energies
  const int M = kern->M;
  for (int d = 0; d < sys->ndev; ++d)
    if (sys->ne[d] > 0 && conv_log2_size(sys->ne[d], M) > 13)
      return fail(ctx, NEGF_ERR_ARG, "device " + std::to_string(d) + ": ne + M must stay <= 8192");
  int max_ne = 0;
  for (int d = 0; d < sys->ndev; ++d) max_ne = std::max(max_ne, (int)sys->ne[d]);
  // workspace after each sweep: the new Sigma^<, Sigma^> ([sum ne nb] blocks each), the
  // kernels, the kernel spectrum and the change statistics
  const size_t sig_bytes = sizeof(zc) * (size_t)nel;
  const size_t need = 2 * sig_bytes + 2 * sizeof(double) * (2 * (size_t)M + 1) + conv_spectrum_bytes(max_ne, M) + 1024;
  if (need > ctx->ws_bytes)
    return fail(ctx, NEGF_ERR_NOMEM, "workspace too small for the self-energy update: needs " + std::to_string(need) +
                                         " bytes");
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaSetDevice(ctx->device));
  negf_scattering sc;
  sc.sigR = sigR_scat;
  sc.sigL = sigL_scat;
  sc.sigL_scale = nullptr;
  sc.per_energy = 1;
  double last = INFINITY;
  int it = 0;
  while (it < max_iter) {
    ++it;
    st = rgf_common(ctx, sys, prec, sigma_L, sigma_R, f_L, f_R, &sc, GR_diag, GR_up, GR_low, GL_diag, GL_low, status, s,
                    true, GG_diag, GG_low);
    if (st != NEGF_OK) return st;
    char* p = (char*)ctx->ws;
    zc* SLn = (zc*)p; p += sig_bytes;
    zc* SGn = (zc*)p; p += sig_bytes;
    double* wl = (double*)p; p += sizeof(double) * (2 * (size_t)M + 1);
    double* wg = (double*)p; p += sizeof(double) * (2 * (size_t)M + 1);
    double* stats = (double*)p; p += 64;
    p = (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
    zc* Wh = (zc*)p;
    CU(cudaMemcpyAsync(wl, kern->w_lesser, sizeof(double) * (2 * (size_t)M + 1), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(wg, kern->w_greater, sizeof(double) * (2 * (size_t)M + 1), cudaMemcpyHostToDevice, s));
    for (int d = 0; d < sys->ndev; ++d) {
      const int ne = sys->ne[d];
      if (ne == 0) continue;
      const long long o4 = Lay.off[8 * (size_t)d + 4];
      const long long per_e = (long long)sys->nb[d] * sys->bs[d] * sys->bs[d];
      ctx->launches += 4;
      CU(energy_convolution((const zc*)GL_diag + o4, SLn + o4, per_e, (int)per_e, ne, M, wl, Wh, s));
      CU(energy_convolution((const zc*)GG_diag + o4, SGn + o4, per_e, (int)per_e, ne, M, wg, Wh, s));
    }
    ++ctx->launches;
    CU(scba_mix((zc*)sigL_scat, (zc*)sigG_scat, (zc*)sigR_scat, SLn, SGn, nel, mixing, stats, s));
    CU(cudaMemcpyAsync(ctx->h_pinned, stats, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    double h[3];
    memcpy(h, ctx->h_pinned, sizeof(h));
    last = std::sqrt(std::max(h[0], h[1])) / std::max(std::sqrt(h[2]), 1e-300);   // the stats are squared
    if (last < tol) break;
  }
  if (iters) *iters = it;
  if (change) *change = last;
  return NEGF_OK;
}

negf_status negf_rgf_arrowhead(negf_ctx* c, const negf_system* sys, negf_precision prec, const void* H_tip,
                               const void* H_arrow, const void* sigma_L, const void* sigma_R,
                               const negf_scattering* scat, void* GR_diag, void* GR_up, void* GR_low, void* G_tip,
                               void* G_row, void* G_col, int32_t* status, negf_stream stream) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  Layout Lay;
  negf_status st = make_layout(ctx, sys, Lay);
  if (st != NEGF_OK) return st;
  if ((st = check_system(ctx, sys)) != NEGF_OK) return st;
  if (prec != NEGF_FP64 && prec != NEGF_MIXED && prec != NEGF_MIXED_TF32)
    return fail(ctx, NEGF_ERR_ARG, "unknown precision");
  if (!H_tip || !H_arrow) return fail(ctx, NEGF_ERR_ARG, "H_tip and H_arrow are required");
  if (!sigma_L || !sigma_R) return fail(ctx, NEGF_ERR_ARG, "sigma_L and sigma_R are required");
  if (!GR_diag || !G_tip || !G_row || !G_col) return fail(ctx, NEGF_ERR_ARG, "GR_diag, G_tip, G_row, G_col are required");
  bool multi = false;
  for (int d = 0; d < sys->ndev; ++d) multi |= sys->nb[d] > 1;
  if (multi && (!GR_up || !GR_low)) return fail(ctx, NEGF_ERR_ARG, "GR_up and GR_low are required when nb > 1");
  if (scat && scat->per_energy != 0 && scat->per_energy != 1)
    return fail(ctx, NEGF_ERR_ARG, "scattering per_energy must be 0 or 1");
  cudaStream_t s = (cudaStream_t)stream;
  CU(cudaSetDevice(ctx->device));
  if (status) CU(cudaMemsetAsync(status, 0, sizeof(int32_t) * Lay.off[8 * (size_t)sys->ndev + 2], s));
  Engine eng{ctx, s, (int)prec, nullptr};
  long long tip_off = 0;   // [sum b*b] offset of this device's tip Hamiltonian
  for (int d = 0; d < sys->ndev; ++d) {
    const int ne = sys->ne[d], nb = sys->nb[d], b = sys->bs[d];
    const long long bb = (long long)b * b;
    const long long* o = &Lay.off[8 * (size_t)d];
    const long long this_tip = tip_off;
    tip_off += bb;
    if (ne == 0) continue;
    const DevView dv = dev_view(sys, Lay, d);
    const ScatView sc = scat_view(scat, Lay, d, nb, b);
    RgfIO io;
    io.sigma_L = (const zc*)sigma_L + o[3];
    io.sigma_R = (const zc*)sigma_R + o[3];
    io.fL = io.fR = nullptr;
    io.GRd = (zc*)GR_diag + o[4];
    io.GRu = GR_up ? (zc*)GR_up + o[5] : nullptr;
    io.GRl = GR_low ? (zc*)GR_low + o[5] : nullptr;
    io.GLd = io.GLl = nullptr;
    io.status = status ? status + o[2] : nullptr;
    io.lesser = false;
    ArrowIO ar;
    ar.H_tip = (const zc*)H_tip + this_tip;
    ar.H_arrow = (const zc*)H_arrow + o[0];
    ar.Gt = (zc*)G_tip + o[3];
    ar.Grow = (zc*)G_row + o[4];
    ar.Gcol = (zc*)G_col + o[4];
    // the device's arrow blocks of A, shared by its energies, ahead of the chunk workspace
    const size_t arrow_bytes = ((2 * sizeof(zc) * (size_t)nb * bb) + 1023) & ~(size_t)1023;
    zc* Arow = (zc*)ctx->ws;
    zc* Acol = Arow + (long long)nb * bb;
    const size_t per = arrowhead_bytes_per_energy(nb, b, eng.mixed);
    const size_t avail = ctx->ws_bytes > arrow_bytes + 2048 ? ctx->ws_bytes - arrow_bytes - 2048 : 0;
    int chunk = (int)std::min<size_t>(avail / per, (size_t)65535);
    if (chunk < 1)
      return fail(ctx, NEGF_ERR_NOMEM, "workspace too small: one energy of this device needs " + std::to_string(per) + " bytes");
    chunk = std::min(chunk, ne);
    ++ctx->launches;
    arrow_blocks_kernel<<<dim3((unsigned)std::min<long long>((bb + 255) / 256, 1024), nb), 256, 0, s>>>(
        Arow, Acol, ar.H_arrow, b);
    CU(cudaGetLastError());
    for (int e0 = 0; e0 < ne; e0 += chunk) {
      const int U = std::min(chunk, ne - e0);
      eng.inv_scratch = nullptr;
      st = rgf_arrowhead_chunk(ctx, eng, dv, sc, io, ar, Arow, Acol, e0, U, (char*)ctx->ws + arrow_bytes + 1024);
      if (st != NEGF_OK) return st;
    }
  }
  return NEGF_OK;
}

negf_status negf_rgf_keldysh(negf_ctx* c, const negf_system* sys, negf_precision prec, const void* sigma_L,
                             const void* sigma_R, const double* f_L, const double* f_R,
                             const negf_scattering* scat, void* GR_diag, void* GR_up, void* GR_low, void* GL_diag,
                             void* GL_low, void* GG_diag, void* GG_low, int32_t* status, negf_stream stream) {
  return rgf_common(reinterpret_cast<Ctx*>(c), sys, prec, sigma_L, sigma_R, f_L, f_R, scat, GR_diag, GR_up,
                    GR_low, GL_diag, GL_low, status, (cudaStream_t)stream, true, GG_diag, GG_low);
}

// ---------------------------------------------------------------------------
negf_status negf_obc(negf_ctx* c, const negf_system* sys, negf_precision prec, double tol, int32_t max_iter,
                     const void* g0_L, const void* g0_R, void* sigma_L, void* sigma_R, void* gs_L, void* gs_R,
                     int32_t* iters, int32_t* newton, int32_t* status, negf_stream stream) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  Layout L;
  negf_status st = make_layout(ctx, sys, L);
  if (st != NEGF_OK) return st;
  if ((st = check_system(ctx, sys)) != NEGF_OK) return st;
  if (!sigma_L || !sigma_R) return fail(ctx, NEGF_ERR_ARG, "sigma_L and sigma_R outputs are required");
  if (!(tol > 0.0) || max_iter < 1 || max_iter > 1000)
    return fail(ctx, NEGF_ERR_ARG, "need tol > 0 and 1 <= max_iter <= 1000");
  if (prec != NEGF_FP64 && prec != NEGF_MIXED && prec != NEGF_MIXED_TF32)
    return fail(ctx, NEGF_ERR_ARG, "unknown precision");
  for (int d = 0; d < sys->ndev; ++d)
    if (sys->nb[d] < 2) return fail(ctx, NEGF_ERR_ARG, "OBC needs nb >= 2 (the lead hop is H_{0,1})");
  CU(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  Engine eng{ctx, s, 0, nullptr};
  const double target = 1e-13;   // Newton target
  const double accept = 1e-10;   // success threshold of the surface residual
  const bool any_warm = g0_L || g0_R;
  // the jobs: a device alone in its block size, or all devices of a block size as one
  // batch of (device, energy) units (work list as in the sweeps)
  std::vector<std::vector<int>> jobs;
  {
    std::vector<int> sizes;
    for (int d = 0; d < sys->ndev; ++d)
      if (sys->ne[d] > 0 && std::find(sizes.begin(), sizes.end(), sys->bs[d]) == sizes.end()) sizes.push_back(sys->bs[d]);
    for (int bsz : sizes) {
      std::vector<int> devs;
      for (int d = 0; d < sys->ndev; ++d)
        if (sys->ne[d] > 0 && sys->bs[d] == bsz) devs.push_back(d);
      jobs.push_back(devs);
    }
  }
  for (const std::vector<int>& devs : jobs) {
    const bool batched = devs.size() > 1;
    const int d = devs[0];
    const DevView dv = dev_view(sys, L, d);
    const long long* o = &L.off[8 * (size_t)d];
    const int b = dv.b;
    const long long bb = (long long)b * b;
    const size_t blk = sizeof(zc) * bb;
    const int nslots = 15;
    std::vector<UnitDev> ud;
    WorkList w;
    std::vector<long long> off_s;   // per unit: its lead block's element offset (o[3] + e b^2)
    int ne = sys->ne[d];
    if (batched) {
      for (int dd : devs) {
        UnitDev x;
        x.dv = dev_view(sys, L, dd);
        ud.push_back(x);
      }
      w = make_worklist(sys, L, devs, bb);
      ne = (int)w.unit_dev.size();
      for (int k = 0; k < ne; ++k) off_s.push_back(L.off[8 * (size_t)devs[w.unit_dev[k]] + 3] + (long long)w.unit_e[k] * bb);
    }
    // products on the sliced tensor-core path (FP64-class) when asked for and supported
    const int sl = (prec == NEGF_MIXED && oz_supported(b)) ? 1 : 0;
    eng.mixed = sl;
    const size_t per_unit = nslots * blk + 96 + zinv_scratch_bytes(b, 1, 0) + (sl ? ozt_scratch_bytes(b, 1) : 0) +
                            (batched ? 3 * sizeof(int) + sizeof(long long) : 0);
    const size_t fixed = 8192 + (batched ? (sizeof(UnitDev) * ud.size() + 6 * 256) : 0);
    if (ctx->ws_bytes <= fixed) return fail(ctx, NEGF_ERR_NOMEM, "workspace too small for one OBC energy");
    int chunk = (int)std::min<size_t>((ctx->ws_bytes - fixed) / (2 * per_unit), (size_t)32767);
    if (chunk < 1) return fail(ctx, NEGF_ERR_NOMEM, "workspace too small for one OBC energy");
    chunk = std::min(chunk, ne);
    for (int e0 = 0; e0 < ne; e0 += chunk) {
      const int U = std::min(chunk, ne - e0);
      const int NU = 2 * U;
      char* p = (char*)ctx->ws;
      // batched: the chunk's unit tables ahead of the slots
      const UnitDev* t_udev = nullptr;
      const int *t_dev = nullptr, *t_e = nullptr, *t_glob = nullptr;
      const long long* t_off = nullptr;
      if (batched) {
        auto put = [&](const void* src, size_t bytes) -> const void* {
          void* dst = p;
          p += (bytes + 255) & ~(size_t)255;
          return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) == cudaSuccess ? dst : nullptr;
        };
        t_udev = (const UnitDev*)put(ud.data(), sizeof(UnitDev) * ud.size());
        t_dev = (const int*)put(w.unit_dev.data() + e0, sizeof(int) * U);
        t_e = (const int*)put(w.unit_e.data() + e0, sizeof(int) * U);
        t_glob = (const int*)put(w.unit_glob.data() + e0, sizeof(int) * U);
        t_off = (const long long*)put(off_s.data() + e0, sizeof(long long) * U);
        if (!t_udev || !t_dev || !t_e || !t_glob || !t_off) return fail(ctx, NEGF_ERR_CUDA, "copying the OBC unit tables failed");
      }
      auto slot = [&]() { zc* q = (zc*)p; p += blk * (size_t)NU; return BMat{q, bb}; };
      BMat a00 = slot(), al0 = slot(), be0 = slot(), eps = slot(), epss = slot(), al = slot(), be = slot();
      BMat g = slot();
      BMat T[7];
      for (int k = 0; k < 7; ++k) T[k] = slot();
      double* ref = (double*)p; p += sizeof(double) * NU;
      double* res = (double*)p; p += sizeof(double) * NU;
      double* resn = (double*)p; p += sizeof(double) * NU;
      long long* coff = (long long*)p; p += sizeof(long long) * NU;   // compact unit list (block offsets)
      int* done = (int*)p; p += sizeof(int) * NU;
      int* it_arr = (int*)p; p += sizeof(int) * NU;
      int* need = (int*)p; p += sizeof(int) * NU;
      int* act = (int*)p; p += sizeof(int) * NU;
      int* warm = (int*)p; p += sizeof(int) * NU;     // unit has a guess
      int* keep = (int*)p; p += sizeof(int) * NU;     // warm result kept
      int* cold = (int*)p; p += sizeof(int) * NU;     // unit goes through the decimation
      int* nsteps = (int*)p; p += sizeof(int) * NU;   // Newton steps taken
      int* redo = (int*)p; p += sizeof(int) * NU;     // refined inverse redone in FP64
      int* n_active = (int*)p; p += 16;
      p = (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
      eng.inv_scratch = zinv_scratch_bytes(b, NU, 0) ? (void*)p : nullptr;
      p += zinv_scratch_bytes(b, NU, 0);
      p = (char*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
      eng.ozt_scratch = sl ? (void*)p : nullptr;

      LeadArgs la{dv, e0, U, a00.p, al0.p, be0.p, eps.p, epss.p, al.p, be.p};
      la.udev = t_udev;
      la.unit_dev = t_dev;
      la.unit_e = t_e;
      dim3 eg((unsigned)std::min<long long>((bb + 255) / 256, 1024), NU);
      lead_init_kernel<<<eg, 256, 0, s>>>(la);
      KCHECK();
      CU(cudaMemsetAsync(nsteps, 0, sizeof(int) * NU, s));
      CU(cudaMemsetAsync(keep, 0, sizeof(int) * NU, s));

      // X = M^{-1} for the units in `mask` (all when NULL), FP64-class.  Mixed: FP32
      // Gauss-Jordan with two refinement steps on the sliced products (residuals in
      // T0, T1), then FP64 Gauss-Jordan for the units whose last residual shows that
      // the refinement did not reach FP64 class (ill-conditioned eps near band edges);
      // FP64 precision: FP64 Gauss-Jordan
      auto lead_inverse = [&](BMat X, BMat M, const int* mask) -> negf_status {
        if (!sl) {
          CU(eng.inv(X, M, b, NU, mask, 0, nullptr));
          return NEGF_OK;
        }
        CU(eng.inverse(X, M, b, NU, nullptr, T[0], T[1], 2, mask));
        refine_check_kernel<<<NU, 256, 0, s>>>(T[0], b, mask, 1e-7, redo);
        KCHECK();
        // units whose refinement converges slowly (kappa(eps) up to ~1e7) take two more
        // steps; FP64 Gauss-Jordan for what is left
        CU(eng.refine_steps(X, M, b, NU, T[0], T[1], 2, redo));
        refine_check_kernel<<<NU, 256, 0, s>>>(T[0], b, redo, 1e-7, redo);
        KCHECK();
        CU(eng.inv(X, M, b, NU, redo, 0, nullptr));
        return NEGF_OK;
      };
      auto residual = [&](BMat X, double* out, const int* mask) -> negf_status {
        CU(eng.gemm(T[0], al0, OP_N, X, OP_N, ONE, NOMAT, ZERO, b, NU, mask));               // al X
        CU(eng.gemm(T[1], T[0], OP_N, be0, OP_N, MONE, a00, ONE, b, NU, mask));              // K = a00 - al X be
        CU(eng.gemm(T[2], T[1], OP_N, X, OP_N, ONE, NOMAT, ZERO, b, NU, mask));              // K X
        residual_kernel<<<NU, 256, 0, s>>>(T[2], b, out, mask);                              // F = K X - I
        KCHECK();
        return NEGF_OK;
      };
      // Products over a compact list of units: the units active at the last count (a
      // superset of those active now, since units only leave the loops; a listed unit
      // that has finished since computes results that are never read again) instead of
      // a launch over all NU units with a mask, once at most half of them are active
      int ncomp = 0;   // > 0: the products run over the list in coff
      auto compact = [&](const int* mask, int cnt) -> negf_status {
        ncomp = 0;
        if (cnt <= 0 || 2 * cnt > NU) return NEGF_OK;
        ++ctx->launches;
        compact_kernel<<<1, 1024, 0, s>>>(mask, NU, bb, coff);
        CU(cudaGetLastError());
        ncomp = cnt;
        return NEGF_OK;
      };
      auto lgemm = [&](BMat D, BMat A, int opA, BMat B, int opB, zc alpha, BMat C, zc beta,
                       const int* mask, bool reuse_a = false) -> cudaError_t {
        if (ncomp > 0) {
          auto cm = [&](BMat m) {
            if (m.p) m.off = coff;
            return m;
          };
          return eng.gemm(cm(D), cm(A), opA, cm(B), opB, alpha, cm(C), beta, b, ncomp, nullptr, reuse_a);
        }
        return eng.gemm(D, A, opA, B, opB, alpha, C, beta, b, NU, mask, reuse_a);
      };
      auto n_set = [&](const int* flags) -> int {
        ++ctx->launches;
        count_kernel<<<1, 256, 0, s>>>(flags, NU, n_active);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_pinned, n_active, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e == cudaSuccess ? ctx->h_pinned[0] : -1;
      };
      // One Newton step on F(X) = (a00 - al X be) X - I for the units flagged in `mask`:
      // K D - al D (be g) = -F, solved as the Stein equation D = -K^{-1}F + (K^{-1} al) D (be g)
      // by Smith doubling (at most 96 levels); gn = g + D and resn = its residual.
      // T1 = K and T2 = F of the current g must be in place (left by the last residual);
      // cnt = the number of units in `mask`.
      auto newton_step = [&](int* mask, BMat gn, int cnt) -> negf_status {
        negf_status sc;
        CU(eng.inv(T[3], T[1], b, NU, mask, 0, nullptr));                 // K^{-1}
        if ((sc = compact(mask, cnt)) != NEGF_OK) return sc;
        CU(lgemm(T[4], T[3], OP_N, al0, OP_N, ONE, NOMAT, ZERO, mask));          // P = K^{-1} al
        CU(lgemm(T[5], be0, OP_N, g, OP_N, ONE, NOMAT, ZERO, mask));             // Q = be g
        CU(lgemm(T[6], T[3], OP_N, T[2], OP_N, MONE, NOMAT, ZERO, mask));        // S = -K^{-1} F
        CU(cudaMemcpyAsync(act, mask, sizeof(int) * NU, cudaMemcpyDeviceToDevice, s));
        BMat Pm = T[4], Qm = T[5], Sm = T[6], W1 = T[0], W2 = T[2], W3 = T[3];
        for (int j = 0; j < 96; ++j) {
          CU(lgemm(W1, Pm, OP_N, Sm, OP_N, ONE, NOMAT, ZERO, act));              // P S
          CU(lgemm(W2, W1, OP_N, Qm, OP_N, ONE, NOMAT, ZERO, act));              // P S Q
          smith_accum_kernel<<<NU, 256, 0, s>>>(Sm, W2, b, act, 1e-15);
          KCHECK();
          CU(lgemm(W1, Pm, OP_N, Pm, OP_N, ONE, NOMAT, ZERO, act));              // P^2
          CU(lgemm(W3, Qm, OP_N, Qm, OP_N, ONE, NOMAT, ZERO, act));              // Q^2
          std::swap(Pm, W1);
          std::swap(Qm, W3);
          balance_kernel<<<NU, 256, 0, s>>>(Pm, Qm, b, act);
          KCHECK();
          if ((j & 7) == 7) {
            const int c2 = n_set(act);
            if (c2 < 0) return fail(ctx, NEGF_ERR_CUDA, "OBC: flag read-back failed");
            if (c2 == 0) break;
            if ((sc = compact(act, c2)) != NEGF_OK) return sc;
          }
        }
        ncomp = 0;
        add_kernel<<<eg, 256, 0, s>>>(gn, g, Sm, b, mask);                                  // g + D
        KCHECK();
        return residual(gn, resn, mask);
      };

      // ---- warm start: Newton from the guesses, kept only if converged and retarded
      if (any_warm) {
        const long long gb = batched ? 0 : o[3] + (long long)e0 * bb;   // batched: per-unit offsets
        const zc* gl = g0_L ? (const zc*)g0_L + gb : nullptr;
        const zc* gr = g0_R ? (const zc*)g0_R + gb : nullptr;
        guess_init_kernel<<<eg, 256, 0, s>>>(g, gl, gr, U, b, warm, t_off);
        KCHECK();
        if ((st = residual(g, res, warm)) != NEGF_OK) return st;
        need_warm_kernel<<<(NU + 255) / 256, 256, 0, s>>>(warm, res, need, NU, target);
        KCHECK();
        for (int step = 0; step < 8; ++step) {
          const int cnt = n_set(need);
          if (cnt < 0) return fail(ctx, NEGF_ERR_CUDA, "OBC: flag read-back failed");
          if (cnt == 0) break;
          if ((st = newton_step(need, eps, cnt)) != NEGF_OK) return st;   // eps is free until the decimation
          newton_take_kernel<<<NU, 256, 0, s>>>(g, eps, b, res, resn, need, target, nsteps);
          KCHECK();
        }
        retarded_check_kernel<<<NU, 256, 0, s>>>(g, T[0], b, warm, res, accept, 1e-12, keep);
        KCHECK();
        lead_init_kernel<<<eg, 256, 0, s>>>(la);   // restore the decimation slots
        KCHECK();
      }
      not_kernel<<<(NU + 255) / 256, 256, 0, s>>>(keep, cold, NU);
      KCHECK();
      const int n_cold = any_warm ? n_set(cold) : NU;
      if (n_cold < 0) return fail(ctx, NEGF_ERR_CUDA, "OBC: flag read-back failed");

      lead_norm_kernel<<<NU, 256, 0, s>>>(al, be, b, 0, ref, done, act, it_arr, 0, tol, n_active, keep);
      KCHECK();
      if (n_cold > 0) {
        // ---- decimation
        for (int it = 0; it <= max_iter; ++it) {
          // counts after the first step (most units end there) and every fourth
          const bool poll = it == 1 || (it & 3) == 3 || it == max_iter;
          if (poll) CU(cudaMemsetAsync(n_active, 0, sizeof(int), s));
          lead_norm_kernel<<<NU, 256, 0, s>>>(al, be, b, 1, ref, done, act, it_arr, it, tol,
                                              poll ? n_active : nullptr);
          KCHECK();
          if (poll) {
            CU(cudaMemcpyAsync(ctx->h_pinned, n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            if (ctx->h_pinned[0] == 0) break;
            if ((st = compact(act, ctx->h_pinned[0])) != NEGF_OK) return st;
          }
          if (it == max_iter) break;
          if ((st = lead_inverse(g, eps, act)) != NEGF_OK) return st;        // g = eps^{-1}
          // the two products of each left operand back to back (the sliced product keeps
          // its digit images for the second)
          CU(lgemm(T[0], al, OP_N, g, OP_N, ONE, NOMAT, ZERO, act));              // al g
          CU(lgemm(T[2], T[0], OP_N, be, OP_N, ONE, NOMAT, ZERO, act));           // al g be
          CU(lgemm(T[4], T[0], OP_N, al, OP_N, MONE, NOMAT, ZERO, act, true));    // -al g al
          CU(lgemm(T[1], be, OP_N, g, OP_N, ONE, NOMAT, ZERO, act));              // be g
          CU(lgemm(T[3], T[1], OP_N, al, OP_N, ONE, NOMAT, ZERO, act));           // be g al
          CU(lgemm(T[5], T[1], OP_N, be, OP_N, MONE, NOMAT, ZERO, act, true));    // -be g be
          lead_update_kernel<<<eg, 256, 0, s>>>(eps, epss, T[2], T[3], b, done);
          KCHECK();
          std::swap(al, T[4]);
          std::swap(be, T[5]);
        }
        ncomp = 0;
        // ---- surface function and its residual
        if ((st = lead_inverse(g, epss, any_warm ? cold : nullptr)) != NEGF_OK) return st;
        if ((st = residual(g, res, any_warm ? cold : nullptr)) != NEGF_OK) return st;
        // ---- Newton polishing of the decimation result above the target
        set_need_kernel<<<(NU + 255) / 256, 256, 0, s>>>(res, need, NU, target, cold);
        KCHECK();
        BMat gn = eps;   // decimation slots are free now
        for (int step = 0; step < 3; ++step) {
          const int cnt = n_set(need);
          if (cnt < 0) return fail(ctx, NEGF_ERR_CUDA, "OBC: flag read-back failed");
          if (cnt == 0) break;
          if ((st = newton_step(need, gn, cnt)) != NEGF_OK) return st;
          newton_accept_kernel<<<NU, 256, 0, s>>>(g, gn, b, res, resn, need, target, nsteps);
          KCHECK();
          // units that took the step continue from T1/T2 (K, F of the accepted g)
        }
      }
      // the lead blocks of the chunk's energies in the outputs: contiguous for one device,
      // at the work list's offsets for a batch
      auto lead_out = [&](void* base) {
        if (batched) return BMat{(zc*)base, 0, 0, 0, t_off};
        return BMat{(zc*)base + o[3] + (long long)e0 * bb, bb};
      };
      if (gs_L) { ++ctx->launches; CU(bcopy(lead_out(gs_L), g, b, U, s)); }
      if (gs_R) { ++ctx->launches; CU(bcopy(lead_out(gs_R), BMat{g.p + (long long)U * bb, bb}, b, U, s)); }
      // sigma = al0 g be0 (left units -> sigma_L, right -> sigma_R)
      CU(eng.gemm(T[0], al0, OP_N, g, OP_N, ONE, NOMAT, ZERO, b, NU));
      CU(eng.gemm(lead_out(sigma_L), T[0], OP_N, be0, OP_N, ONE, NOMAT, ZERO, b, U));
      CU(eng.gemm(lead_out(sigma_R), BMat{T[0].p + (long long)U * bb, bb}, OP_N,
                  BMat{be0.p + (long long)U * bb, bb}, OP_N, ONE, NOMAT, ZERO, b, U));
      const long long ob = batched ? 0 : o[2] + e0;   // batched: per-unit energy indices
      obc_finish_kernel<<<(U + 127) / 128, 128, 0, s>>>(
          done, res, it_arr, nsteps, U, status ? status + ob : nullptr, iters ? iters + 2 * ob : nullptr,
          newton ? newton + 2 * ob : nullptr, accept, t_glob);
      KCHECK();
    }
  }
  return NEGF_OK;
}

negf_status negf_observables(negf_ctx* c, const negf_system* sys, negf_precision prec, const void* sigma_L,
                             const double* e_weight,
                             const void* GR_diag, const void* GR_up, const void* GR_low, const void* GL_diag,
                             const void* GL_low, double* T, double* dos, double* current, double* density,
                             negf_stream stream) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  Layout L;
  negf_status st = make_layout(ctx, sys, L);
  if (st != NEGF_OK) return st;
  if ((st = check_system(ctx, sys)) != NEGF_OK) return st;
  const bool overlap = sys->S_up != nullptr;
  if (T && (!sigma_L || !GR_diag)) return fail(ctx, NEGF_ERR_ARG, "T needs sigma_L and GR_diag");
  if (dos && (!GR_diag || (overlap && (!GR_up || !GR_low))))
    return fail(ctx, NEGF_ERR_ARG, "DOS needs GR_diag (and GR_up, GR_low when S_up is given)");
  if (current && !GL_low) return fail(ctx, NEGF_ERR_ARG, "current needs GL_low");
  if (density && (!GL_diag || !e_weight || (overlap && !GL_low)))
    return fail(ctx, NEGF_ERR_ARG, "density needs GL_diag, e_weight (and GL_low when S_up is given)");
  if (prec != NEGF_FP64 && prec != NEGF_MIXED && prec != NEGF_MIXED_TF32)
    return fail(ctx, NEGF_ERR_ARG, "unknown precision");
  CU(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  Engine eng{ctx, s, 0, nullptr};
  if (density) CU(cudaMemsetAsync(density, 0, sizeof(double) * L.off[8 * (size_t)sys->ndev + 7], s));
  for (int d = 0; d < sys->ndev; ++d) {
    const int ne = sys->ne[d];
    if (ne == 0) continue;
    const DevView dv = dev_view(sys, L, d);
    const long long* o = &L.off[8 * (size_t)d];
    const int sl = (T && prec == NEGF_MIXED && oz_supported(dv.b)) ? 1 : 0;
    const size_t per = observables_bytes_per_energy(dv, sl);
    const size_t avail = ctx->ws_bytes > 4096 ? ctx->ws_bytes - 4096 : 0;
    int chunk = (int)std::min<size_t>(avail / per, (size_t)65535);
    if (chunk < 1) return fail(ctx, NEGF_ERR_NOMEM, "workspace too small for one energy");
    chunk = std::min(chunk, ne);
    ObsIO ob;
    ob.sigma_L = sigma_L ? (const zc*)sigma_L + o[3] : nullptr;
    ob.w = e_weight ? e_weight + o[2] : nullptr;
    ob.GRd = GR_diag ? (const zc*)GR_diag + o[4] : nullptr;
    ob.GRu = GR_up ? (const zc*)GR_up + o[5] : nullptr;
    ob.GRl = GR_low ? (const zc*)GR_low + o[5] : nullptr;
    ob.GLd = GL_diag ? (const zc*)GL_diag + o[4] : nullptr;
    ob.GLl = GL_low ? (const zc*)GL_low + o[5] : nullptr;
    ob.T = T ? T + o[2] : nullptr;
    ob.dos = dos ? dos + o[2] : nullptr;
    ob.current = current ? current + o[6] : nullptr;
    ob.density = density ? density + o[7] : nullptr;
    for (int e0 = 0; e0 < ne; e0 += chunk) {
      const int U = std::min(chunk, ne - e0);
      if ((st = observables_chunk(ctx, eng, dv, ob, sl, e0, U, 0, (char*)ctx->ws)) != NEGF_OK) return st;
    }
  }
  return NEGF_OK;
}

negf_status negf_rgf_observables(negf_ctx* c, const negf_system* sys, negf_precision prec, const void* sigma_L,
                                 const void* sigma_R, const double* f_L, const double* f_R,
                                 const negf_scattering* scat, const double* e_weight, double* T, double* dos,
                                 double* current, double* density, int32_t* status, negf_stream stream) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  Layout L;
  negf_status st = make_layout(ctx, sys, L);
  if (st != NEGF_OK) return st;
  if ((st = check_system(ctx, sys)) != NEGF_OK) return st;
  if (prec != NEGF_FP64 && prec != NEGF_MIXED && prec != NEGF_MIXED_TF32)
    return fail(ctx, NEGF_ERR_ARG, "unknown precision");
  if (!sigma_L || !sigma_R || !f_L || !f_R) return fail(ctx, NEGF_ERR_ARG, "lead self-energies and occupations required");
  if (density && !e_weight) return fail(ctx, NEGF_ERR_ARG, "density needs e_weight");
  if (scat && scat->per_energy != 0 && scat->per_energy != 1)
    return fail(ctx, NEGF_ERR_ARG, "scattering per_energy must be 0 or 1");
  CU(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (status) CU(cudaMemsetAsync(status, 0, sizeof(int32_t) * L.off[8 * (size_t)sys->ndev + 2], s));
  if (density) CU(cudaMemsetAsync(density, 0, sizeof(double) * L.off[8 * (size_t)sys->ndev + 7], s));
  Engine eng{ctx, s, (int)prec, nullptr};
  for (int d = 0; d < sys->ndev; ++d) {
    const int ne = sys->ne[d];
    if (ne == 0) continue;
    const DevView dv = dev_view(sys, L, d);
    const ScatView sc = scat_view(scat, L, d, dv.nb, dv.b);
    const long long* o = &L.off[8 * (size_t)d];
    const int nb = dv.nb, b = dv.b;
    const long long bb = (long long)b * b;
    const size_t blk = sizeof(zc) * (size_t)bb;
    // per energy: its G^R / G^< blocks (diagonal, upper, lower; diagonal, lower), the sweep
    // workspace and the observables' scratch
    const size_t gblocks = (size_t)(2 * nb + 3 * std::max(nb - 1, 0));
    RgfIO io;
    io.sigma_L = (const zc*)sigma_L + o[3];
    io.sigma_R = (const zc*)sigma_R + o[3];
    io.fL = f_L + o[2];
    io.fR = f_R + o[2];
    io.status = status ? status + o[2] : nullptr;
    io.lesser = true;
    // outputs go to per-chunk buffers (non-null here only so that the sizing below counts
    // no sweep-internal storage for them; set per chunk)
    io.GRd = io.GRu = io.GRl = io.GLd = io.GLl = (zc*)ctx->ws;
    const int sl = (T && prec == NEGF_MIXED && oz_supported(b)) ? 1 : 0;
    const size_t per = gblocks * blk + rgf_bytes_per_energy(nb, b, io, eng.mixed) + observables_bytes_per_energy(dv, sl) + 3072;
    // the device's W blocks ahead of the chunks, when there is room for them next to one energy
    const size_t wb = asm_w_bytes(nb, b);
    const bool use_w = ctx->ws_bytes >= wb + per;
    int chunk = (int)std::min<size_t>((ctx->ws_bytes - (use_w ? wb : 0)) / per, (size_t)65535);
    if (chunk < 1)
      return fail(ctx, NEGF_ERR_NOMEM, "workspace too small: one energy of this device needs " + std::to_string(per) + " bytes");
    chunk = std::min(chunk, ne);
    io.W = nullptr;
    if (use_w) {
      zc* W = (zc*)ctx->ws;
      ++ctx->launches;
      asm_w_kernel<<<dim3((unsigned)std::min<long long>((bb + 255) / 256, 1024), nb), 256, 0, s>>>(
          dv, W, W + nb * bb, W + (2LL * nb - 1) * bb);
      CU(cudaGetLastError());
      io.W = W;
    }
    for (int e0 = 0; e0 < ne; e0 += chunk) {
      const int U = std::min(chunk, ne - e0);
      char* p = (char*)ctx->ws + (use_w ? wb : 0);
      auto take = [&](size_t nblocks) { zc* q = (zc*)p; p += blk * nblocks * (size_t)U; return q; };
      io.GRd = take(nb);
      io.GLd = take(nb);
      io.GRu = nb > 1 ? take(nb - 1) : nullptr;
      io.GRl = nb > 1 ? take(nb - 1) : nullptr;
      io.GLl = nb > 1 ? take(nb - 1) : nullptr;
      p = (char*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
      eng.inv_scratch = nullptr;
      if ((st = rgf_chunk(ctx, eng, dv, sc, io, e0, U, p, nullptr, e0)) != NEGF_OK) return st;   // buffers start at e0
      // the observables' scratch after the sweep's workspace (the sweep is done with it)
      char* q = p + (size_t)U * rgf_bytes_per_energy(nb, b, io, eng.mixed);
      q = (char*)(((uintptr_t)q + 1023) & ~(uintptr_t)1023);
      ObsIO ob;
      ob.sigma_L = (const zc*)sigma_L + o[3];
      ob.w = e_weight ? e_weight + o[2] : nullptr;
      ob.GRd = io.GRd; ob.GRu = io.GRu; ob.GRl = io.GRl; ob.GLd = io.GLd; ob.GLl = io.GLl;
      ob.T = T ? T + o[2] : nullptr;
      ob.dos = dos ? dos + o[2] : nullptr;
      ob.current = current ? current + o[6] : nullptr;
      ob.density = density ? density + o[7] : nullptr;
      Engine eo{ctx, s, 0, nullptr};
      if ((st = observables_chunk(ctx, eo, dv, ob, sl, e0, U, e0, q)) != NEGF_OK) return st;
    }
  }
  return NEGF_OK;
}

negf_status negf_profile_enable(negf_ctx* c, int enable) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  ctx->prof = enable != 0;
  return NEGF_OK;
}

negf_status negf_profile_read(negf_ctx* c, int64_t* launches, int64_t* k_launches, double* k_ms, double* k_flops,
                              double* k_bytes) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  CU(cudaSetDevice(ctx->device));
  for (const ProfRec& r : ctx->recs) {
    CU(cudaEventSynchronize(r.ev1));
    float ms = 0.f;
    CU(cudaEventElapsedTime(&ms, r.ev0, r.ev1));
    ctx->k_launches[r.cls] += 1;
    ctx->k_ms[r.cls] += ms;
    ctx->k_flops[r.cls] += r.flops;
    ctx->k_bytes[r.cls] += r.bytes;
    ctx->pool.push_back(r.ev0);
    ctx->pool.push_back(r.ev1);
  }
  ctx->recs.clear();
  if (launches) *launches = ctx->launches;
  for (int k = 0; k < K_NCLASS; ++k) {
    if (k_launches) k_launches[k] = ctx->k_launches[k];
    if (k_ms) k_ms[k] = ctx->k_ms[k];
    if (k_flops) k_flops[k] = ctx->k_flops[k];
    if (k_bytes) k_bytes[k] = ctx->k_bytes[k];
  }
  return NEGF_OK;
}

negf_status negf_selftest_wait_timeout(negf_ctx* c, int64_t wait_ns, negf_stream stream) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  if (wait_ns < 1000000 || wait_ns > 2000000000)
    return fail(ctx, NEGF_ERR_ARG, "wait_ns must lie in [1e6, 2e9]");
  CU(cudaSetDevice(ctx->device));
  ++ctx->launches;
  CU(wait_selftest(ctx->d_err, (unsigned long long)wait_ns, (cudaStream_t)stream));
  return NEGF_OK;
}

negf_status negf_profile_reset(negf_ctx* c) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  int64_t dummy;
  negf_status st = negf_profile_read(c, &dummy, nullptr, nullptr, nullptr, nullptr);
  if (st != NEGF_OK) return st;
  ctx->launches = 0;
  for (int k = 0; k < K_NCLASS; ++k) {
    ctx->k_launches[k] = 0; ctx->k_ms[k] = 0; ctx->k_flops[k] = 0; ctx->k_bytes[k] = 0;
  }
  return NEGF_OK;
}

negf_status negf_block_gemm(negf_ctx* c, negf_precision prec, int32_t n, int32_t units, int32_t opA, int32_t opB,
                            const double* alpha, const void* A, int64_t a_stride, const void* B, int64_t b_stride,
                            const double* beta, const void* C, int64_t c_stride, void* D, int64_t d_stride,
                            negf_stream stream) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  if (n < 1 || n > 4096 || units < 0 || units > 65535) return fail(ctx, NEGF_ERR_ARG, "need 1 <= n <= 4096, 0 <= units <= 65535");
  if ((opA != OP_N && opA != OP_H) || (opB != OP_N && opB != OP_H)) return fail(ctx, NEGF_ERR_ARG, "op must be 0 or 2");
  if (!alpha || !A || !B || !D || (C && !beta)) return fail(ctx, NEGF_ERR_ARG, "NULL operand");
  if (prec != NEGF_FP64 && prec != NEGF_MIXED && prec != NEGF_MIXED_TF32)
    return fail(ctx, NEGF_ERR_ARG, "unknown precision");
  if (a_stride < 0 || b_stride < 0 || c_stride < 0 || d_stride < 0) return fail(ctx, NEGF_ERR_ARG, "negative stride");
  if (d_stride == 0 && units > 1) return fail(ctx, NEGF_ERR_ARG, "D cannot be shared by several units");
  CU(cudaSetDevice(ctx->device));
  Engine eng{ctx, (cudaStream_t)stream, (int)prec, nullptr};
  if (oz_scratch_bytes(n, units) > ctx->ws_bytes) return fail(ctx, NEGF_ERR_NOMEM, "workspace too small");
  if (ozt_scratch_bytes(n, units) <= ctx->ws_bytes) eng.ozt_scratch = ctx->ws;
  else eng.oz_scratch = ctx->ws;
  CU(eng.gemm(BMat{(zc*)D, d_stride}, BMat{(zc*)A, a_stride}, opA, BMat{(zc*)B, b_stride}, opB,
              zmake(alpha[0], alpha[1]), C ? BMat{(zc*)C, c_stride} : NOMAT,
              C ? zmake(beta[0], beta[1]) : ZERO, n, units));
  return NEGF_OK;
}

// random complex entries in [-1, 1) from a counter-based hash (splitmix64 of the index)
__global__ void fill_random_kernel(zc* x, long long n, unsigned long long seed) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const double re = (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    const double im = (double)((z << 11) >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    x[i] = zmake(re, im);
  }
}

negf_status negf_tune_products(negf_ctx* c, int32_t n, int32_t units, int32_t* choice, double* ms,
                               negf_stream stream) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  if (n < 1 || n > 512 || units < 1 || units > 65535) return fail(ctx, NEGF_ERR_ARG, "need 1 <= n <= 512, 1 <= units <= 65535");
  if (!oz_supported(n)) {   // no sliced product for this n: nothing to choose
    if (choice) *choice = OZ_DEFAULT;
    if (ms) for (int v = 0; v < OZ_NVARIANT; ++v) ms[v] = -1.0;
    return NEGF_OK;
  }
  const long long nn = (long long)n * n;
  const size_t mats = sizeof(zc) * (size_t)nn * units;
  const size_t need = 3 * mats + 1024 + ozt_scratch_bytes(n, units);
  if (need > ctx->ws_bytes) return fail(ctx, NEGF_ERR_NOMEM, "workspace too small to tune " + std::to_string(units) + " units");
  CU(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  zc* A = (zc*)ctx->ws;
  zc* B = A + nn * units;
  zc* D = B + nn * units;
  void* scratch = (void*)(((uintptr_t)(D + nn * units) + 1023) & ~(uintptr_t)1023);
  ctx->launches += 2;
  fill_random_kernel<<<1024, 256, 0, s>>>(A, nn * units, 20260101ull);
  fill_random_kernel<<<1024, 256, 0, s>>>(B, nn * units, 20260202ull);
  CU(cudaGetLastError());
  GemmArgs g;
  g.D = BMat{D, nn}; g.A = BMat{A, nn}; g.B = BMat{B, nn}; g.C = BMat{nullptr, 0};
  g.opA = OP_N; g.opB = OP_N; g.alpha = zmake(1.0, 0.0); g.beta = zmake(0.0, 0.0);
  g.n = n; g.units = units; g.active = nullptr;
  cudaEvent_t e0 = ctx->take_event(), e1 = ctx->take_event();
  int best = OZ_DEFAULT;
  double best_ms = INFINITY;
  for (int v = OZ_HALF; v < OZ_NVARIANT; ++v) {
    if (ms) ms[v] = -1.0;
    if (!oz_variant_supported(n, v)) continue;
    CU(zgemm_ozt_variant(g, scratch, ctx->d_err, s, v));   // warm-up
    CU(cudaEventRecord(e0, s));
    constexpr int reps = 3;
    for (int r = 0; r < reps; ++r) CU(zgemm_ozt_variant(g, scratch, ctx->d_err, s, v));
    CU(cudaEventRecord(e1, s));
    CU(cudaEventSynchronize(e1));
    float t = 0.f;
    CU(cudaEventElapsedTime(&t, e0, e1));
    const double per = (double)t / reps;
    ctx->launches += 2 * (reps + 1);
    if (ms) ms[v] = per;
    if (per < best_ms) { best_ms = per; best = v; }
  }
  ctx->pool.push_back(e0);
  ctx->pool.push_back(e1);
  if (ms) ms[OZ_DEFAULT] = -1.0;
  ctx->oz_variant[n] = best;
  if (choice) *choice = best;
  return NEGF_OK;
}

negf_status negf_set_product_variant(negf_ctx* c, int32_t n, int32_t variant) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  if (n < 1 || n > 512) return fail(ctx, NEGF_ERR_ARG, "need 1 <= n <= 512");
  if (variant < 0 || variant >= OZ_NVARIANT || (variant != OZ_DEFAULT && !oz_variant_supported(n, variant)))
    return fail(ctx, NEGF_ERR_ARG, "variant " + std::to_string(variant) + " does not support n = " + std::to_string(n));
  ctx->oz_variant[n] = variant;
  return NEGF_OK;
}

negf_status negf_block_inverse(negf_ctx* c, negf_precision prec, int32_t n, int32_t units, const void* M, void* X,
                               int32_t* status, negf_stream stream) {
  Ctx* ctx = reinterpret_cast<Ctx*>(c);
  if (!ctx) return fail(nullptr, NEGF_ERR_ARG, "ctx is NULL");
  if (n < 1 || n > 512 || units < 0) return fail(ctx, NEGF_ERR_ARG, "need 1 <= n <= 512, units >= 0");
  if (!M || !X) return fail(ctx, NEGF_ERR_ARG, "NULL operand");
  if (prec != NEGF_FP64 && prec != NEGF_MIXED && prec != NEGF_MIXED_TF32)
    return fail(ctx, NEGF_ERR_ARG, "unknown precision");
  if (units == 0) return NEGF_OK;
  CU(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int mixed = (int)prec;
  const long long bb = (long long)n * n;
  // workspace: two scratch slots for the refinement, the inverse scratch, the product scales
  const size_t inv_b = zinv_scratch_bytes(n, units, mixed ? 1 : 0);
  const size_t need = (size_t)units * bb * sizeof(zc) * (mixed ? 2 : 0) + inv_b + oz_scratch_bytes(n, units);
  if (need > ctx->ws_bytes) return fail(ctx, NEGF_ERR_NOMEM, "workspace too small for this batch of inverses");
  zc* ws = (zc*)ctx->ws;
  Engine eng{ctx, s, mixed, nullptr};
  BMat T1{ws, bb}, T2{ws + (mixed ? units * bb : 0), bb};
  eng.inv_scratch = (void*)(ws + (mixed ? 2 * units * bb : 0));
  eng.oz_scratch = (char*)eng.inv_scratch + inv_b;
  {
    char* q = (char*)(((uintptr_t)eng.oz_scratch + 1023) & ~(uintptr_t)1023);
    if ((size_t)(q - (char*)ctx->ws) + ozt_scratch_bytes(n, units) <= ctx->ws_bytes) eng.ozt_scratch = q;
  }
  if (status) CU(cudaMemsetAsync(status, 0, sizeof(int32_t) * units, s));
  CU(eng.inverse(BMat{(zc*)X, bb}, BMat{(zc*)M, bb}, n, units, status, T1, T2));
  return NEGF_OK;
}

}  // extern "C"

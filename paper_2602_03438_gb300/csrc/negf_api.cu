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
  zc *Adiag, *Aup, *Alow, *SigL;   // slot bases (unit stride b*b), each nullable
  zc* SigG;                        // Sigma^>_ii slot (nullable)
  const zc *sigma_L, *sigma_R;     // lead self-energies of this device, [ne] blocks
  const double *fL, *fR;           // this device's occupations (nullable unless SigL)
};

// One 32 x 32 tile of every requested block per CTA (32 x 8 threads, 4 rows each);
// the conjugate-transposed terms (A_{j+1,j}, the lead Gamma's Sigma^H) are read as the
// transposed tile through shared memory, so that every global access is a row segment.
constexpr int ASM_T = 32;

__global__ void __launch_bounds__(256) assemble_kernel(AsmArgs a) {
  const int u = blockIdx.y;
  const int b = a.dv.b, nb = a.dv.nb;
  const long long bb = (long long)b * b;
  const int e = a.e0 + u;
  const zc z = zmake(a.dv.E[e], a.dv.eta);
  const int ntile = (b + ASM_T - 1) / ASM_T;
  const int r0 = (blockIdx.x / ntile) * ASM_T, c0 = (blockIdx.x % ntile) * ASM_T;
  const int tx = threadIdx.x, ty = threadIdx.y;
  __shared__ zc tS[ASM_T][ASM_T + 1], tH[ASM_T][ASM_T + 1];
  const int i = a.i_diag, j = a.i_off;
  const bool lead_lesser = (a.SigL || a.SigG) && (i == 0 || i == nb - 1);
  const zc* sg = (i == 0) ? a.sigma_L + e * bb : a.sigma_R + e * bb;
  const double fo = (i == 0) ? (a.fL ? a.fL[e] : 0.0) : (a.fR ? a.fR[e] : 0.0);
  // transposed tiles: (row c0 + ty + 8k, column r0 + tx) of S_up, H_up (for A_{j+1,j}) and
  // of the lead Sigma (for Sigma^H), stored as [tx][ty + 8k]
  if (a.Alow) {
#pragma unroll
    for (int k = 0; k < ASM_T / 8; ++k) {
      const int rr = c0 + ty + 8 * k, cc = r0 + tx;
      zc sv = zmake(0.0, 0.0), hv = zmake(0.0, 0.0);
      if (rr < b && cc < b) {
        if (a.dv.Su) sv = a.dv.Su[j * bb + (long long)rr * b + cc];
        hv = a.dv.Hu[j * bb + (long long)rr * b + cc];
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
      zc s = a.dv.Sd ? a.dv.Sd[i * bb + rc] : zmake(r == c ? 1.0 : 0.0, 0.0);
      zc v = zsub(zmul(z, s), a.dv.Hd[i * bb + rc]);
      if (a.sc.sigR) v = zsub(v, a.sc.sigR[e * a.sc.e_stride + i * bb + rc]);
      if (i == 0) v = zsub(v, a.sigma_L[e * bb + rc]);
      if (i == nb - 1) v = zsub(v, a.sigma_R[e * bb + rc]);
      a.Adiag[u * bb + rc] = v;
    }
    if (a.Aup) {   // A_{j,j+1} = z S_up - H_up
      zc s = a.dv.Su ? a.dv.Su[j * bb + rc] : zmake(0.0, 0.0);
      a.Aup[u * bb + rc] = zsub(zmul(z, s), a.dv.Hu[j * bb + rc]);
    }
    if (a.Alow) {  // A_{j+1,j} = z S_up^H - H_up^H: element (r, c) = conj of (c, r)
      const zc s = zconj(tS[ty + 8 * k][tx]);
      a.Alow[u * bb + rc] = zsub(zmul(z, s), zconj(tH[ty + 8 * k][tx]));
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
  assemble_kernel<<<dim3((unsigned)(nt * nt), a.units), dim3(ASM_T, 8), 0, s>>>(a);
  return cudaGetLastError();
}

// D = D - W + W^H   (the anti-Hermitian completion of G^<_ii)
__global__ void antiherm_update_kernel(BMat D, BMat W, int n) {
  const int u = blockIdx.y;
  const long long nn = (long long)n * n;
  zc* d = D.at(u);
  const zc* w = W.at(u);
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nn;
       idx += (long long)gridDim.x * blockDim.x) {
    const int r = (int)(idx / n), c = (int)(idx - (long long)r * n);
    d[idx] = zadd(zsub(d[idx], w[idx]), zconj(w[(long long)c * n + r]));
  }
}

cudaError_t antiherm_update(BMat D, BMat W, int n, int units, cudaStream_t s) {
  if (units <= 0) return cudaSuccess;
  const long long nn = (long long)n * n;
  dim3 grid((unsigned)std::min<long long>((nn + 255) / 256, 1024), units);
  antiherm_update_kernel<<<grid, 256, 0, s>>>(D, W, n);
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
__global__ void one_minus_kernel(BMat R, int n) {
  const int u = blockIdx.y;
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
  cudaError_t sliced(const GemmArgs& g) {
    return ozt_scratch ? zgemm_ozt(g, ozt_scratch, ctx->d_err, s) : zgemm_oz(g, oz_scratch, ctx->d_err, s);
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
  cudaError_t gemm(BMat D, BMat A, int opA, BMat B, int opB, zc alpha, BMat C, zc beta, int n, int units,
                   const int* active = nullptr) {
    GemmArgs g;
    g.D = D; g.A = A; g.B = B; g.C = C;
    g.opA = opA; g.opB = opB; g.alpha = alpha; g.beta = beta;
    g.n = n; g.units = units; g.active = active;
    const double nn = (double)n * n;
    const double flops = 8.0 * nn * n * units;                        // useful complex flops
    const double bytes = 16.0 * nn * units * (3.0 + (C.p ? 1.0 : 0.0));   // A, B, D (+C) once each
    cudaError_t e;
    const bool masked = active != nullptr;   // masked launches do an unknown share of the work
    if (mixed == 1 && can_slice(n)) {
      begin(masked ? K_OTHER : K_GEMM_OZ);
      e = sliced(g);
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
    const bool masked = active != nullptr;   // masked launches do an unknown share of the work
    begin(masked ? K_OTHER : (single ? K_INV_F32 : K_INV_F64));
    cudaError_t e = zinv(X, M, n, units, active, single, inv_scratch, status, s);
    end(masked ? 0.0 : 8.0 * (double)n * n * n * units, masked ? 0.0 : 32.0 * (double)n * n * units);
    return e;
  }
  // X = M^{-1}.  Mixed precision: FP32 Gauss-Jordan, then `refine` steps of
  // X <- X + X (I - M X) with the residual I - M X formed in FP64 and the
  // correction product on the engine's GEMM.  T1, T2: scratch slots.
  // Refinement steps: two with the sliced product (each step squares the relative
  // error of the FP32 inverse, so kappa ~ 1e6 blocks need two), one with the TF32 mode.
  cudaError_t inverse(BMat X, BMat M, int n, int units, int32_t* status, BMat T1, BMat T2, int refine = -1) {
    if (refine < 0) refine = (mixed == 1) ? 2 : 1;
    cudaError_t e = inv(X, M, n, units, nullptr, mixed ? 1 : 0, status);
    if (e != cudaSuccess || !mixed) return e;
    const long long nn = (long long)n * n;
    dim3 grid((unsigned)std::min<long long>((nn + 255) / 256, 1024), units);
    for (int k = 0; k < refine; ++k) {
      GemmArgs r;
      r.D = T1; r.A = M; r.B = X; r.C = BMat{nullptr, 0};
      r.opA = OP_N; r.opB = OP_N; r.alpha = zmake(1.0, 0.0); r.beta = zmake(0.0, 0.0);
      r.n = n; r.units = units; r.active = nullptr;
      // M X with FP64-class accuracy: the sliced tensor-core product, else FP64 FMA
      if (mixed == 1 && can_slice(n)) {
        begin(K_GEMM_OZ);
        e = sliced(r);
      } else {
        begin(K_GEMM_F64);
        e = zgemm_f64(r, s);
      }
      end(8.0 * (double)n * n * n * units, 48.0 * (double)n * n * units);
      if (e != cudaSuccess) return e;
      ++ctx->launches;
      one_minus_kernel<<<grid, 256, 0, s>>>(T1, n);                        // I - M X
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      if (mixed == 1 && ozt_scratch && oz_supported(n)) {
        // X <- X + X (I - M X) in one product: these kernels read op(A) only through the
        // digit images made before they start, and C and D element by element in one
        // thread, so D, A and C may all be X
        if ((e = gemm(X, X, OP_N, T1, OP_N, zmake(1.0, 0.0), X, zmake(1.0, 0.0), n, units)) != cudaSuccess)
          return e;
        continue;
      }
      if ((e = gemm(T2, X, OP_N, T1, OP_N, zmake(1.0, 0.0), BMat{nullptr, 0}, zmake(0.0, 0.0), n, units)) !=
          cudaSuccess)
        return e;                                                          // X (I - M X)
      ++ctx->launches;
      add_kernel<<<grid, 256, 0, s>>>(X, X, T2, n, nullptr);
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
};

negf_status rgf_chunk(Ctx* ctx, Engine& eng, const DevView& dv, const ScatView& sc, const RgfIO& io, int e0,
                      int U, char* ws) {
  const int nb = dv.nb, b = dv.b;
  const long long bb = (long long)b * b;
  const size_t blk = sizeof(zc) * bb;
  cudaStream_t s = eng.s;
  // ---- workspace slots (each U blocks, unit stride b*b)
  char* p = ws;
  auto slot = [&](int count) { zc* q = (zc*)p; p += blk * (size_t)U * count; return q; };
  zc* Adiag = slot(1);
  zc* Aup = slot(1);
  zc* Alow = slot(1);
  zc* SigL = io.lesser ? slot(1) : nullptr;
  const bool greater = io.lesser && io.greater;
  zc* SigG = greater ? slot(1) : nullptr;
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

  auto S1 = [&](zc* base) { return BMat{base, bb}; };
  // per-energy output blocks: [e][i] with unit stride nb*b*b (diag) or (nb-1)*b*b (off-diagonal)
  auto gD = [&](int i) {
    return io.GRd ? BMat{io.GRd + ((long long)e0 * nb + i) * bb, (long long)nb * bb}
                  : BMat{gbase + (long long)i * U * bb, bb};
  };
  auto glD = [&](int i) {
    return io.GLd ? BMat{io.GLd + ((long long)e0 * nb + i) * bb, (long long)nb * bb}
                  : BMat{glbase + (long long)i * U * bb, bb};
  };
  auto ggD = [&](int i) {
    return io.GGd ? BMat{io.GGd + ((long long)e0 * nb + i) * bb, (long long)nb * bb}
                  : BMat{ggbase + (long long)i * U * bb, bb};
  };
  auto Yb = [&](int i) { return BMat{Ybase + (long long)i * U * bb, bb}; };
  // the Keldysh kinds of this call: G^< and, with `greater`, G^> (the same recursion on
  // Sigma^> in place of Sigma^<)
  struct Kind { zc* sig; std::function<BMat(int)> D; zc* low; };
  std::vector<Kind> kinds;
  if (io.lesser) kinds.push_back(Kind{SigL, glD, io.GLl});
  if (greater) kinds.push_back(Kind{SigG, ggD, io.GGl});
  auto offB = [&](zc* base, int i) { return BMat{base + ((long long)e0 * (nb - 1) + i) * bb, (long long)(nb - 1) * bb}; };

  AsmArgs a;
  a.dv = dv; a.sc = sc; a.e0 = e0; a.units = U;
  a.sigma_L = io.sigma_L; a.sigma_R = io.sigma_R; a.fL = io.fL; a.fR = io.fR;
  int32_t* st = io.status ? io.status + e0 : nullptr;

  // ---------------- forward sweep
  for (int i = 0; i < nb; ++i) {
    a.i_diag = i;
    a.i_off = i - 1;
    a.Adiag = Adiag; a.SigL = SigL; a.SigG = SigG;
    a.Aup = (i > 0) ? Aup : nullptr;
    a.Alow = (i > 0) ? Alow : nullptr;
    ++ctx->launches;
    CU(assemble(a, s));
    if (i == 0) {
      CU(eng.inverse(gD(0), S1(Adiag), b, U, st, S1(T[1]), S1(T[2])));
      for (const Kind& k : kinds) {
        CU(eng.gemm(S1(T[2]), gD(0), OP_N, S1(k.sig), OP_N, ONE, NOMAT, ZERO, b, U));
        CU(eng.gemm(k.D(0), S1(T[2]), OP_N, gD(0), OP_H, ONE, NOMAT, ZERO, b, U));
      }
      continue;
    }
    // Y_{i-1} = A_{i,i-1} g_{i-1};  M = A_ii - Y_{i-1} A_{i-1,i};  g_i = M^{-1}
    CU(eng.gemm(Yb(i - 1), S1(Alow), OP_N, gD(i - 1), OP_N, ONE, NOMAT, ZERO, b, U));
    CU(eng.gemm(S1(T[0]), Yb(i - 1), OP_N, S1(Aup), OP_N, MONE, S1(Adiag), ONE, b, U));
    CU(eng.inverse(gD(i), S1(T[0]), b, U, st, S1(T[1]), S1(T[2])));
    for (const Kind& k : kinds) {
      // g^x_i = g_i (Sigma^x_ii + A_{i,i-1} g^x_{i-1} A_{i,i-1}^H) g_i^H   (x = <, >)
      CU(eng.gemm(S1(T[1]), S1(Alow), OP_N, k.D(i - 1), OP_N, ONE, NOMAT, ZERO, b, U));
      CU(eng.gemm(S1(T[2]), S1(T[1]), OP_N, S1(Alow), OP_H, ONE, S1(k.sig), ONE, b, U));
      CU(eng.gemm(S1(T[3]), gD(i), OP_N, S1(T[2]), OP_N, ONE, NOMAT, ZERO, b, U));
      CU(eng.gemm(k.D(i), S1(T[3]), OP_N, gD(i), OP_H, ONE, NOMAT, ZERO, b, U));
    }
  }
  // ---------------- backward sweep
  a.Adiag = nullptr; a.SigL = nullptr; a.SigG = nullptr;
  for (int i = nb - 2; i >= 0; --i) {
    a.i_diag = -1;
    a.i_off = i;
    a.Aup = Aup; a.Alow = Alow;
    ++ctx->launches;
    CU(assemble(a, s));
    const BMat X = S1(T[0]);
    const BMat Gup = io.GRu ? offB(io.GRu, i) : S1(gup_tmp);
    // X = g_i A_{i,i+1};  G_{i,i+1} = -X G_{i+1,i+1};  G_ii = g_i - G_{i,i+1} Y_i;  G_{i+1,i} = -G_{i+1,i+1} Y_i
    CU(eng.gemm(X, gD(i), OP_N, S1(Aup), OP_N, ONE, NOMAT, ZERO, b, U));
    CU(eng.gemm(Gup, X, OP_N, gD(i + 1), OP_N, MONE, NOMAT, ZERO, b, U));
    CU(eng.gemm(gD(i), Gup, OP_N, Yb(i), OP_N, MONE, gD(i), ONE, b, U));
    if (io.GRl) CU(eng.gemm(offB(io.GRl, i), gD(i + 1), OP_N, Yb(i), OP_N, MONE, NOMAT, ZERO, b, U));
    for (const Kind& k : kinds) {
      const BMat Z = S1(T[1]), P = S1(T[2]), Wm = S1(T[3]);
      // Z = A_{i+1,i} g^x_i;  P = G^x_{i+1,i+1} X^H;  W = G_{i,i+1} Z   (x = <, >)
      CU(eng.gemm(Z, S1(Alow), OP_N, k.D(i), OP_N, ONE, NOMAT, ZERO, b, U));
      CU(eng.gemm(P, k.D(i + 1), OP_N, X, OP_H, ONE, NOMAT, ZERO, b, U));
      CU(eng.gemm(Wm, Gup, OP_N, Z, OP_N, ONE, NOMAT, ZERO, b, U));
      // G^x_ii = g^x_i + X P - W + W^H
      CU(eng.gemm(k.D(i), X, OP_N, P, OP_N, ONE, k.D(i), ONE, b, U));
      ++ctx->launches;
      CU(antiherm_update(k.D(i), Wm, b, U, s));
      // G^x_{i+1,i} = -G_{i+1,i+1} Z - P
      if (k.low) CU(eng.gemm(offB(k.low, i), gD(i + 1), OP_N, Z, OP_N, MONE, P, MONE, b, U));
    }
  }
  return NEGF_OK;
}

size_t rgf_bytes_per_energy(int nb, int b, const RgfIO& io, int mixed) {
  const size_t blk = sizeof(zc) * (size_t)b * b;
  const bool greater = io.lesser && io.greater;
  size_t n = 3 + (io.lesser ? 1 : 0) + (greater ? 1 : 0) + 4 + std::max(nb - 1, 1);
  if (!io.GRd) n += nb;
  if (io.lesser && !io.GLd) n += nb;
  if (greater && !io.GGd) n += nb;
  if (!io.GRu) n += 1;
  size_t bytes = n * blk;
  bytes += zinv_scratch_bytes(b, 1, mixed ? 1 : 0);
  if (mixed == 1) bytes += ozt_scratch_bytes(b, 1) + 1024;
  return bytes;
}

// ---------------------------------------------------------------------------
// OBC: decimation + Newton polishing, FP64, units = (side, energy)
// ---------------------------------------------------------------------------
struct LeadArgs {
  DevView dv;
  int e0, U;
  zc *a00, *al0, *be0, *eps, *epss, *al, *be;   // slot bases, unit stride b*b, 2U units
};

// unit u < U: left lead of energy e0+u; u >= U: right lead of energy e0+u-U
__global__ void lead_init_kernel(LeadArgs a) {
  const int u = blockIdx.y;
  const int b = a.dv.b, nb = a.dv.nb;
  const long long bb = (long long)b * b;
  const bool left = u < a.U;
  const int e = a.e0 + (left ? u : u - a.U);
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
  double m = 0.0;
  for (long long i = threadIdx.x; i < nn; i += blockDim.x) {
    m = fmax(m, hypot(x[i].x, x[i].y));
    m = fmax(m, hypot(y[i].x, y[i].y));
  }
  __shared__ double red[32];
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
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

// Smith step bookkeeping: S += inc; conv if max|inc| <= tol max|S|; rebalance P, Q
__global__ void smith_accum_kernel(BMat S, BMat inc, int n, int* act, double tol) {
  const int u = blockIdx.x;
  if (!act[u]) return;
  const long long nn = (long long)n * n;
  zc* s = S.at(u);
  const zc* d = inc.at(u);
  double mi = 0.0, ms = 0.0;
  for (long long i = threadIdx.x; i < nn; i += blockDim.x) {
    zc v = zadd(s[i], d[i]);
    s[i] = v;
    mi = fmax(mi, hypot(d[i].x, d[i].y));
    ms = fmax(ms, hypot(v.x, v.y));
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
    if (mi <= tol * fmax(ms, 1e-300) || !isfinite(ms)) act[u] = 0;
  }
}

__global__ void balance_kernel(BMat P, BMat Q, int n, const int* act) {
  const int u = blockIdx.x;
  if (!act[u]) return;
  const long long nn = (long long)n * n;
  zc* p = P.at(u);
  zc* q = Q.at(u);
  double mp = 0.0, mq = 0.0;
  for (long long i = threadIdx.x; i < nn; i += blockDim.x) {
    mp = fmax(mp, hypot(p[i].x, p[i].y));
    mq = fmax(mq, hypot(q[i].x, q[i].y));
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
    sc = (mp > 0.0 && mq > 0.0) ? sqrt(mq / mp) : 1.0;
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
__global__ void guess_init_kernel(BMat g, const zc* g0L, const zc* g0R, int U, int n, int* warm) {
  const int u = blockIdx.y;
  const bool left = u < U;
  const zc* src = left ? g0L : g0R;
  if (blockIdx.x == 0 && threadIdx.x == 0) warm[u] = src ? 1 : 0;
  if (!src) return;
  const long long nn = (long long)n * n;
  src += (long long)(left ? u : u - U) * nn;
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
                                  int32_t* status, int32_t* iters_out, int32_t* newton_out, double accept) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= U) return;
  const bool okL = done[e] == 1 && res[e] <= accept;
  const bool okR = done[U + e] == 1 && res[U + e] <= accept;
  if (status) status[e] = (okL && okR) ? NEGF_OK : NEGF_ERR_NOCONV;
  if (iters_out) {
    iters_out[2 * e] = iters[e];
    iters_out[2 * e + 1] = iters[U + e];
  }
  if (newton_out) {
    newton_out[2 * e] = nsteps[e];
    newton_out[2 * e + 1] = nsteps[U + e];
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

// DOS(E) = -(1/pi) Im Tr[G S] over the BT pattern, one CTA per energy
__global__ void dos_kernel(DevView dv, const zc* GRd, const zc* GRu, const zc* GRl, int e0, double* dos) {
  const int u = blockIdx.x, e = e0 + u;
  const int nb = dv.nb, b = dv.b;
  const long long bb = (long long)b * b;
  double acc = 0.0;   // accumulates Im Tr[G S]
  for (int i = 0; i < nb; ++i) {
    const zc* g = GRd + ((long long)e * nb + i) * bb;
    if (!dv.Sd) {
      for (int r = threadIdx.x; r < b; r += blockDim.x) acc += g[(long long)r * b + r].y;
    } else {
      const zc* S = dv.Sd + i * bb;
#pragma unroll 4
      for (long long k = threadIdx.x; k < bb; k += blockDim.x) {   // sum_pq G_pq S_qp
        const int p = (int)(k / b), q = (int)(k - (long long)p * b);
        const zc v = zmul(g[k], S[(long long)q * b + p]);
        acc += v.y;
      }
    }
  }
  if (dv.Su && GRu && GRl) {
    for (int i = 0; i + 1 < nb; ++i) {
      const zc* gu = GRu + ((long long)e * (nb - 1) + i) * bb;
      const zc* gl = GRl + ((long long)e * (nb - 1) + i) * bb;
      const zc* Su = dv.Su + i * bb;
#pragma unroll 4
      for (long long k = threadIdx.x; k < bb; k += blockDim.x) {
        const int p = (int)(k / b), q = (int)(k - (long long)p * b);
        // G_{i,i+1}[p][q] S_{i+1,i}[q][p] with S_{i+1,i} = S_up^H: S_{i+1,i}[q][p] = conj(Su[p][q])
        acc += zmul(gu[k], zconj(Su[k])).y;
        // G_{i+1,i}[p][q] S_{i,i+1}[q][p]
        acc += zmul(gl[k], Su[(long long)q * b + p]).y;
      }
    }
  }
  __shared__ double red[32];
  const double t = block_sum<256>(acc, red);
  if (threadIdx.x == 0) dos[e] = -t / M_PI;
}

// J_i(E) = 2 Re Tr[(H_{i,i+1} - z S_{i,i+1}) G^<_{i+1,i}], one CTA per (energy, interface)
__global__ void current_kernel(DevView dv, const zc* GLl, int e0, double* J) {
  const int u = blockIdx.y, e = e0 + u, i = blockIdx.x;
  const int nb = dv.nb, b = dv.b;
  const long long bb = (long long)b * b;
  const zc z = zmake(dv.E[e], dv.eta);
  const zc* g = GLl + ((long long)e * (nb - 1) + i) * bb;
  const zc* H = dv.Hu + i * bb;
  const zc* S = dv.Su ? dv.Su + i * bb : nullptr;
  double acc = 0.0;
  // sum_pq A[p][q] G[q][p] with k running along G (coalesced reads of the per-energy block;
  // A = H - z S is shared by all energies and read transposed from L2)
#pragma unroll 4
  for (long long k = threadIdx.x; k < bb; k += blockDim.x) {
    const int q = (int)(k / b), p = (int)(k - (long long)q * b);
    const long long t = (long long)p * b + q;
    zc x = H[t];
    if (S) x = zsub(x, zmul(z, S[t]));
    acc += zmul(x, g[k]).x;
  }
  __shared__ double red[32];
  const double t = block_sum<256>(acc, red);
  if (threadIdx.x == 0) J[(long long)e * (nb - 1) + i] = 2.0 * t;
}

// per-energy orbital occupation Re(-i (G^< S)_kk)/(2 pi) into nE[u][k], k over nb*b
__global__ void density_energy_kernel(DevView dv, const zc* GLd, const zc* GLl, int e0, double* nE) {
  const int u = blockIdx.y, e = e0 + u;
  const int nb = dv.nb, b = dv.b;
  const long long bb = (long long)b * b;
  const long long N = (long long)nb * b;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < N; k += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(k / b), r = (int)(k - (long long)i * b);
    const zc* gd = GLd + ((long long)e * nb + i) * bb;
    zc m;
    if (!dv.Sd) {
      m = gd[(long long)r * b + r];
    } else {
      m = zmake(0.0, 0.0);
      const zc* S = dv.Sd + i * bb;
      for (int l = 0; l < b; ++l) zfma(m, gd[(long long)r * b + l], S[(long long)l * b + r]);
      if (i + 1 < nb) {   // G^<_{i,i+1} S_{i+1,i},  G^<_{i,i+1}[r][l] = -conj(G^<_{i+1,i}[l][r]),  S_{i+1,i}[l][r] = conj(Su[r][l])
        const zc* gl = GLl + ((long long)e * (nb - 1) + i) * bb;
        const zc* Su = dv.Su + i * bb;
        for (int l = 0; l < b; ++l) {
          const zc a = zscale(zconj(gl[(long long)l * b + r]), -1.0);
          zfma(m, a, zconj(Su[(long long)r * b + l]));
        }
      }
      if (i > 0) {        // G^<_{i,i-1} S_{i-1,i}
        const zc* gl = GLl + ((long long)e * (nb - 1) + (i - 1)) * bb;
        const zc* Su = dv.Su + (i - 1) * bb;
        for (int l = 0; l < b; ++l) zfma(m, gl[(long long)r * b + l], Su[(long long)l * b + r]);
      }
    }
    nE[(long long)u * N + k] = m.y / (2.0 * M_PI);   // Re(-i m) = Im m
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

negf_status negf_layout(const negf_system* sys, int64_t* out) {
  if (!out) return fail(nullptr, NEGF_ERR_ARG, "out is NULL");
  Layout L;
  negf_status st = make_layout(nullptr, sys, L);
  if (st != NEGF_OK) return st;
  for (size_t k = 0; k < L.off.size(); ++k) out[k] = L.off[k];
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
  for (int d = 0; d < sys->ndev; ++d) {
    const int ne = sys->ne[d];
    if (ne == 0) continue;
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
    int chunk = (int)std::min<size_t>(ctx->ws_bytes / per, (size_t)65535);
    if (chunk < 1)
      return fail(ctx, NEGF_ERR_NOMEM, "workspace too small: one energy of this device needs " +
                                           std::to_string(per) + " bytes");
    chunk = std::min(chunk, ne);
    for (int e0 = 0; e0 < ne; e0 += chunk) {
      const int U = std::min(chunk, ne - e0);
      eng.inv_scratch = nullptr;
      st = rgf_chunk(ctx, eng, dv, sc, io, e0, U, (char*)ctx->ws);
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
  for (int d = 0; d < sys->ndev; ++d) {
    const int ne = sys->ne[d];
    if (ne == 0) continue;
    const DevView dv = dev_view(sys, L, d);
    const long long* o = &L.off[8 * (size_t)d];
    const int b = dv.b;
    const long long bb = (long long)b * b;
    const size_t blk = sizeof(zc) * bb;
    const int nslots = 15;
    // products on the sliced tensor-core path (FP64-class) when asked for and supported
    const int sl = (prec == NEGF_MIXED && oz_supported(b)) ? 1 : 0;
    eng.mixed = sl;
    const size_t per_unit = nslots * blk + 64 + zinv_scratch_bytes(b, 1, 0) + (sl ? ozt_scratch_bytes(b, 1) : 0);
    int chunk = (int)std::min<size_t>((ctx->ws_bytes - 8192) / (2 * per_unit), (size_t)32767);
    if (chunk < 1) return fail(ctx, NEGF_ERR_NOMEM, "workspace too small for one OBC energy");
    chunk = std::min(chunk, ne);
    for (int e0 = 0; e0 < ne; e0 += chunk) {
      const int U = std::min(chunk, ne - e0);
      const int NU = 2 * U;
      char* p = (char*)ctx->ws;
      auto slot = [&]() { zc* q = (zc*)p; p += blk * (size_t)NU; return BMat{q, bb}; };
      BMat a00 = slot(), al0 = slot(), be0 = slot(), eps = slot(), epss = slot(), al = slot(), be = slot();
      BMat g = slot();
      BMat T[7];
      for (int k = 0; k < 7; ++k) T[k] = slot();
      double* ref = (double*)p; p += sizeof(double) * NU;
      double* res = (double*)p; p += sizeof(double) * NU;
      double* resn = (double*)p; p += sizeof(double) * NU;
      int* done = (int*)p; p += sizeof(int) * NU;
      int* it_arr = (int*)p; p += sizeof(int) * NU;
      int* need = (int*)p; p += sizeof(int) * NU;
      int* act = (int*)p; p += sizeof(int) * NU;
      int* warm = (int*)p; p += sizeof(int) * NU;     // unit has a guess
      int* keep = (int*)p; p += sizeof(int) * NU;     // warm result kept
      int* cold = (int*)p; p += sizeof(int) * NU;     // unit goes through the decimation
      int* nsteps = (int*)p; p += sizeof(int) * NU;   // Newton steps taken
      int* n_active = (int*)p; p += 16;
      p = (char*)(((uintptr_t)p + 255) & ~(uintptr_t)255);
      eng.inv_scratch = zinv_scratch_bytes(b, NU, 0) ? (void*)p : nullptr;
      p += zinv_scratch_bytes(b, NU, 0);
      p = (char*)(((uintptr_t)p + 1023) & ~(uintptr_t)1023);
      eng.ozt_scratch = sl ? (void*)p : nullptr;

      LeadArgs la{dv, e0, U, a00.p, al0.p, be0.p, eps.p, epss.p, al.p, be.p};
      dim3 eg((unsigned)std::min<long long>((bb + 255) / 256, 1024), NU);
      lead_init_kernel<<<eg, 256, 0, s>>>(la);
      KCHECK();
      CU(cudaMemsetAsync(nsteps, 0, sizeof(int) * NU, s));
      CU(cudaMemsetAsync(keep, 0, sizeof(int) * NU, s));

      auto residual = [&](BMat X, double* out, const int* mask) -> negf_status {
        CU(eng.gemm(T[0], al0, OP_N, X, OP_N, ONE, NOMAT, ZERO, b, NU, mask));               // al X
        CU(eng.gemm(T[1], T[0], OP_N, be0, OP_N, MONE, a00, ONE, b, NU, mask));              // K = a00 - al X be
        CU(eng.gemm(T[2], T[1], OP_N, X, OP_N, ONE, NOMAT, ZERO, b, NU, mask));              // K X
        residual_kernel<<<NU, 256, 0, s>>>(T[2], b, out, mask);                              // F = K X - I
        KCHECK();
        return NEGF_OK;
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
      // T1 = K and T2 = F of the current g must be in place (left by the last residual).
      auto newton_step = [&](int* mask, BMat gn) -> negf_status {
        CU(eng.inv(T[3], T[1], b, NU, mask, 0, nullptr));                 // K^{-1}
        CU(eng.gemm(T[4], T[3], OP_N, al0, OP_N, ONE, NOMAT, ZERO, b, NU, mask));          // P = K^{-1} al
        CU(eng.gemm(T[5], be0, OP_N, g, OP_N, ONE, NOMAT, ZERO, b, NU, mask));             // Q = be g
        CU(eng.gemm(T[6], T[3], OP_N, T[2], OP_N, MONE, NOMAT, ZERO, b, NU, mask));        // S = -K^{-1} F
        CU(cudaMemcpyAsync(act, mask, sizeof(int) * NU, cudaMemcpyDeviceToDevice, s));
        BMat Pm = T[4], Qm = T[5], Sm = T[6], W1 = T[0], W2 = T[2], W3 = T[3];
        for (int j = 0; j < 96; ++j) {
          CU(eng.gemm(W1, Pm, OP_N, Sm, OP_N, ONE, NOMAT, ZERO, b, NU, act));              // P S
          CU(eng.gemm(W2, W1, OP_N, Qm, OP_N, ONE, NOMAT, ZERO, b, NU, act));              // P S Q
          smith_accum_kernel<<<NU, 256, 0, s>>>(Sm, W2, b, act, 1e-15);
          KCHECK();
          CU(eng.gemm(W1, Pm, OP_N, Pm, OP_N, ONE, NOMAT, ZERO, b, NU, act));              // P^2
          CU(eng.gemm(W3, Qm, OP_N, Qm, OP_N, ONE, NOMAT, ZERO, b, NU, act));              // Q^2
          std::swap(Pm, W1);
          std::swap(Qm, W3);
          balance_kernel<<<NU, 256, 0, s>>>(Pm, Qm, b, act);
          KCHECK();
          if ((j & 7) == 7) {
            const int cnt = n_set(act);
            if (cnt < 0) return fail(ctx, NEGF_ERR_CUDA, "OBC: flag read-back failed");
            if (cnt == 0) break;
          }
        }
        add_kernel<<<eg, 256, 0, s>>>(gn, g, Sm, b, mask);                                  // g + D
        KCHECK();
        return residual(gn, resn, mask);
      };

      // ---- warm start: Newton from the guesses, kept only if converged and retarded
      if (any_warm) {
        const zc* gl = g0_L ? (const zc*)g0_L + o[3] + (long long)e0 * bb : nullptr;
        const zc* gr = g0_R ? (const zc*)g0_R + o[3] + (long long)e0 * bb : nullptr;
        guess_init_kernel<<<eg, 256, 0, s>>>(g, gl, gr, U, b, warm);
        KCHECK();
        if ((st = residual(g, res, warm)) != NEGF_OK) return st;
        need_warm_kernel<<<(NU + 255) / 256, 256, 0, s>>>(warm, res, need, NU, target);
        KCHECK();
        for (int step = 0; step < 8; ++step) {
          const int cnt = n_set(need);
          if (cnt < 0) return fail(ctx, NEGF_ERR_CUDA, "OBC: flag read-back failed");
          if (cnt == 0) break;
          if ((st = newton_step(need, eps)) != NEGF_OK) return st;   // eps is free until the decimation
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
          const bool poll = (it & 3) == 3 || it == max_iter;
          if (poll) CU(cudaMemsetAsync(n_active, 0, sizeof(int), s));
          lead_norm_kernel<<<NU, 256, 0, s>>>(al, be, b, 1, ref, done, act, it_arr, it, tol,
                                              poll ? n_active : nullptr);
          KCHECK();
          if (poll) {
            CU(cudaMemcpyAsync(ctx->h_pinned, n_active, sizeof(int), cudaMemcpyDeviceToHost, s));
            CU(cudaStreamSynchronize(s));
            if (ctx->h_pinned[0] == 0) break;
          }
          if (it == max_iter) break;
          CU(eng.inv(g, eps, b, NU, act, 0, nullptr));                     // g = eps^{-1}
          CU(eng.gemm(T[0], al, OP_N, g, OP_N, ONE, NOMAT, ZERO, b, NU, act));              // al g
          CU(eng.gemm(T[1], be, OP_N, g, OP_N, ONE, NOMAT, ZERO, b, NU, act));              // be g
          CU(eng.gemm(T[2], T[0], OP_N, be, OP_N, ONE, NOMAT, ZERO, b, NU, act));           // al g be
          CU(eng.gemm(T[3], T[1], OP_N, al, OP_N, ONE, NOMAT, ZERO, b, NU, act));           // be g al
          lead_update_kernel<<<eg, 256, 0, s>>>(eps, epss, T[2], T[3], b, done);
          KCHECK();
          CU(eng.gemm(T[4], T[0], OP_N, al, OP_N, MONE, NOMAT, ZERO, b, NU, act));          // -al g al
          CU(eng.gemm(T[5], T[1], OP_N, be, OP_N, MONE, NOMAT, ZERO, b, NU, act));          // -be g be
          std::swap(al, T[4]);
          std::swap(be, T[5]);
        }
        // ---- surface function and its residual
        CU(eng.inv(g, epss, b, NU, any_warm ? cold : nullptr, 0, nullptr));
        if ((st = residual(g, res, any_warm ? cold : nullptr)) != NEGF_OK) return st;
        // ---- Newton polishing of the decimation result above the target
        set_need_kernel<<<(NU + 255) / 256, 256, 0, s>>>(res, need, NU, target, cold);
        KCHECK();
        BMat gn = eps;   // decimation slots are free now
        for (int step = 0; step < 3; ++step) {
          const int cnt = n_set(need);
          if (cnt < 0) return fail(ctx, NEGF_ERR_CUDA, "OBC: flag read-back failed");
          if (cnt == 0) break;
          if ((st = newton_step(need, gn)) != NEGF_OK) return st;
          newton_accept_kernel<<<NU, 256, 0, s>>>(g, gn, b, res, resn, need, target, nsteps);
          KCHECK();
          // units that took the step continue from T1/T2 (K, F of the accepted g)
        }
      }
      if (gs_L)
        CU(cudaMemcpyAsync((zc*)gs_L + o[3] + (long long)e0 * bb, g.p, blk * U, cudaMemcpyDeviceToDevice, s));
      if (gs_R)
        CU(cudaMemcpyAsync((zc*)gs_R + o[3] + (long long)e0 * bb, g.p + (long long)U * bb, blk * U,
                           cudaMemcpyDeviceToDevice, s));
      // sigma = al0 g be0 (left units -> sigma_L, right -> sigma_R)
      CU(eng.gemm(T[0], al0, OP_N, g, OP_N, ONE, NOMAT, ZERO, b, NU));
      zc* sL = (zc*)sigma_L + o[3] + (long long)e0 * bb;
      zc* sR = (zc*)sigma_R + o[3] + (long long)e0 * bb;
      CU(eng.gemm(BMat{sL, bb}, T[0], OP_N, be0, OP_N, ONE, NOMAT, ZERO, b, U));
      CU(eng.gemm(BMat{sR, bb}, BMat{T[0].p + (long long)U * bb, bb}, OP_N,
                  BMat{be0.p + (long long)U * bb, bb}, OP_N, ONE, NOMAT, ZERO, b, U));
      obc_finish_kernel<<<(U + 127) / 128, 128, 0, s>>>(
          done, res, it_arr, nsteps, U, status ? status + o[2] + e0 : nullptr,
          iters ? iters + 2 * (o[2] + e0) : nullptr, newton ? newton + 2 * (o[2] + e0) : nullptr, accept);
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
    const int b = dv.b, nb = dv.nb;
    const long long bb = (long long)b * b;
    const long long N = (long long)nb * b;
    // T's products on the sliced tensor-core path (FP64-class) when asked for and supported;
    // their scales and digit images follow Gamma, K1 and K2 in the workspace
    const int sl = (T && prec == NEGF_MIXED && oz_supported(b)) ? 1 : 0;
    eng.mixed = sl;
    const size_t per = std::max<size_t>(sizeof(zc) * (size_t)bb * 4 + (sl ? ozt_scratch_bytes(b, 1) : 0),
                                        sizeof(double) * (size_t)N);
    const size_t avail = ctx->ws_bytes > 4096 ? ctx->ws_bytes - 4096 : 0;
    int chunk = (int)std::min<size_t>(avail / per, (size_t)65535);
    if (chunk < 1) return fail(ctx, NEGF_ERR_NOMEM, "workspace too small for one energy");
    chunk = std::min(chunk, ne);
    for (int e0 = 0; e0 < ne; e0 += chunk) {
      const int U = std::min(chunk, ne - e0);
      if (T) {
        zc* p = (zc*)ctx->ws;
        BMat Gam{p, bb}, K1{p + (long long)U * bb, bb}, K2{p + 2LL * U * bb, bb};
        eng.ozt_scratch = sl ? (void*)(((uintptr_t)(p + 3LL * U * bb) + 1023) & ~(uintptr_t)1023) : nullptr;
        BMat Sg{(zc*)sigma_L + o[3] + (long long)e0 * bb, bb};
        BMat G00{(zc*)GR_diag + o[4] + (long long)e0 * nb * bb, (long long)nb * bb};
        dim3 eg((unsigned)std::min<long long>((bb + 255) / 256, 1024), U);
        gamma_kernel<<<eg, 256, 0, s>>>(Gam, Sg, b);
        KCHECK();
        CU(eng.gemm(K1, Gam, OP_N, G00, OP_N, ONE, NOMAT, ZERO, b, U));
        CU(eng.gemm(K2, G00, OP_N, Gam, OP_N, ONE, NOMAT, ZERO, b, U));
        transmission_kernel<<<U, 256, 0, s>>>(Gam, G00, K1, K2, b, T + o[2] + e0);
        KCHECK();
      }
      if (dos) {
        dos_kernel<<<U, 256, 0, s>>>(dv, (const zc*)GR_diag + o[4], GR_up ? (const zc*)GR_up + o[5] : nullptr,
                                     GR_low ? (const zc*)GR_low + o[5] : nullptr, e0, dos + o[2]);
        KCHECK();
      }
      if (current && nb > 1) {
        current_kernel<<<dim3(nb - 1, U), 256, 0, s>>>(dv, (const zc*)GL_low + o[5], e0, current + o[6]);
        KCHECK();
      }
      if (density) {
        double* nE = (double*)ctx->ws;
        dim3 g1((unsigned)std::min<long long>((N + 255) / 256, 1024), U);
        density_energy_kernel<<<g1, 256, 0, s>>>(dv, (const zc*)GL_diag + o[4],
                                                 GL_low ? (const zc*)GL_low + o[5] : nullptr, e0, nE);
        KCHECK();
        density_accum_kernel<<<(unsigned)std::min<long long>((N + 255) / 256, 1024), 256, 0, s>>>(
            nE, e_weight + o[2], e0, U, N, density + o[7]);
        KCHECK();
      }
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

// The RGF sweeps of devices with small blocks (b <= 16) as ONE persistent launch: one CTA
// per energy runs the whole forward and backward recursion of G^R and of the Keldysh
// functions G^< (and G^>) (Sec. II, Eqs. (1)-(2); the textbook block recursion), keeping
// the left-connected blocks and the running G blocks in shared memory, in FP64.
//
// At these sizes every block product is below the smallest tensor-core tile, and the
// batched per-step launches (about 16 launches per block index) are bound by launch and
// fill latency rather than by arithmetic: one CTA per energy with one thread per block
// element does the same FP64 operations with no launch between them.
//
// Forward, i = 0 .. nb-1 (Y_{i-1} = A_{i,i-1} g_{i-1}):
//   g_i = (A_ii - Y_{i-1} A_{i-1,i})^{-1},
//   g^x_i = g_i (Sigma^x_ii + A_{i,i-1} g^x_{i-1} A_{i,i-1}^H) g_i^H          (x = <, >)
// Backward, i = nb-2 .. 0 (X = g_i A_{i,i+1}):
//   G_{i,i+1} = -X G_{i+1,i+1},  G_ii = g_i - G_{i,i+1} Y_i,  G_{i+1,i} = -G_{i+1,i+1} Y_i,
//   Z = A_{i+1,i} g^x_i,  P = G^x_{i+1,i+1} X^H,  W = G_{i,i+1} Z,
//   G^x_ii = g^x_i + X P - W + W^H,  G^x_{i+1,i} = -G_{i+1,i+1} Z - P.
// The block inverse is Gauss-Jordan with partial pivoting (first row of largest
// modulus), in place, its row interchanges undone as column interchanges.
#include "negf_internal.cuh"

namespace negf {

namespace {

constexpr int kSmallB = 16;
constexpr int kSmallThreads = kSmallB * kSmallB;
constexpr int kBufs = 13;

// thread (r, c) owns element (r, c) of every b x b block in shared memory (row stride
// ld = b + 1); a product op(A) op(B) is computed into a register by each owner, and the
// callers synchronise the CTA before a block that others still read is overwritten
struct Prod {
  int b, ld, r, c;
  bool on;   // this thread owns element (r, c)
  __device__ zc mul(const zc* A, bool hA, const zc* B, bool hB) const {
    zc acc = zmake(0.0, 0.0);
    if (!on) return acc;
    for (int k = 0; k < b; ++k) {
      const zc a = hA ? zconj(A[k * ld + r]) : A[r * ld + k];
      const zc v = hB ? zconj(B[c * ld + k]) : B[k * ld + c];
      zfma(acc, a, v);
    }
    return acc;
  }
  __device__ zc get(const zc* A) const { return on ? A[r * ld + c] : zmake(0.0, 0.0); }
  __device__ void put(zc* D, zc v) const {
    if (on) D[r * ld + c] = v;
  }
};

__device__ __forceinline__ void load_blk(zc* dst, const zc* src, const Prod& t) {
  if (t.on) dst[t.r * t.ld + t.c] = src[t.r * t.b + t.c];
}
__device__ __forceinline__ void store_blk(zc* dst, zc v, const Prod& t) {
  if (t.on) dst[t.r * t.b + t.c] = v;
}

// W <- W^{-1} in place (Gauss-Jordan, partial pivoting); returns false (to every thread)
// when a pivot column is zero or not finite
__device__ bool gj_inverse(zc* W, const Prod& t, int* piv, zc* s_dinv, int* s_p, int* s_sing) {
  const int n = t.b, ld = t.ld, tid = threadIdx.x;
  if (tid == 0) *s_sing = 0;
  for (int k = 0; k < n; ++k) {
    if (tid < 32) {
      double best = -1.0;
      int bi = n;
      if (tid >= k && tid < n) {
        best = zabs2(W[tid * ld + k]);
        bi = tid;
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const double ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (tid == 0) {
        if (!(best > 0.0)) { *s_sing = 1; bi = k; }
        *s_p = bi;
        piv[k] = bi;
        const zc d = W[bi * ld + k];
        const double den = zabs2(d);
        *s_dinv = (den > 0.0) ? zmake(d.x / den, -d.y / den) : zmake(0.0, 0.0);
      }
    }
    __syncthreads();
    const int p = *s_p;
    const zc dinv = *s_dinv;
    zc nv = zmake(0.0, 0.0);
    if (t.on) {
      // row r of the interchanged matrix is row src of W
      const int src = (t.r == k) ? p : ((t.r == p) ? k : t.r);
      const zc prc = zmul(W[p * ld + t.c], dinv);   // the scaled pivot row, column c
      if (t.r == k) {
        nv = (t.c == k) ? dinv : prc;
      } else {
        const zc f = W[src * ld + k];
        nv = (t.c == k) ? zmake(-(f.x * dinv.x - f.y * dinv.y), -(f.x * dinv.y + f.y * dinv.x))
                        : zsub(W[src * ld + t.c], zmul(f, prc));
      }
    }
    __syncthreads();
    t.put(W, nv);
    __syncthreads();
  }
  // undo the interchanges: swap columns k and piv[k], last pivot first
  for (int k = n - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k && tid < n) {
      const zc a = W[tid * ld + k];
      W[tid * ld + k] = W[tid * ld + p];
      W[tid * ld + p] = a;
    }
    __syncthreads();
  }
  return *s_sing == 0;
}

__global__ void __launch_bounds__(kSmallThreads) rgf_small_kernel(SmallSweep a) {
  const int u = blockIdx.x;
  const int b = a.b, nb = a.nb;
  const long long bb = (long long)b * b;
  const long long step = (long long)a.U * bb;   // stride of the assembled blocks' index
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = b + 1;
  zc* buf[kBufs];
  for (int q = 0; q < kBufs; ++q) buf[q] = reinterpret_cast<zc*>(smem_raw) + (size_t)q * b * ld;
  __shared__ int piv[kSmallB];
  __shared__ zc s_dinv;
  __shared__ int s_p, s_sing;
  Prod t;
  t.b = b; t.ld = ld;
  t.r = threadIdx.x / b; t.c = threadIdx.x - t.r * b;
  t.on = threadIdx.x < bb;
  bool ok = true;

  // named roles; G/M and the kinds' running blocks swap by index
  zc *Al = buf[0], *Au = buf[1], *Yb = buf[2], *T1 = buf[3], *T2 = buf[4], *S = buf[5];
  zc *X = buf[6], *Gu = buf[7], *P = buf[8];
  int iG = 9, iM = 10;
  zc* K[2] = {buf[11], buf[12]};
  const zc* sigx[2] = {a.Sl, a.Sg};
  const SBlk outx[2] = {a.gL, a.gG};
  const SBlk lowx[2] = {a.Ll, a.Gl};

  // ---------------- forward sweep
  for (int i = 0; i < nb; ++i) {
    zc* M = buf[iM];
    zc* G = buf[iG];   // g_{i-1}
    load_blk(M, a.Ad + i * step + u * bb, t);
    if (i > 0) {
      load_blk(Al, a.Al + (i - 1) * step + u * bb, t);
      load_blk(Au, a.Au + (i - 1) * step + u * bb, t);
    }
    __syncthreads();
    if (i > 0) {
      const zc y = t.mul(Al, false, G, false);   // Y_{i-1} = A_{i,i-1} g_{i-1}
      t.put(Yb, y);
      store_blk(a.Y.at(u, i - 1), y, t);
      __syncthreads();
      const zc m = zsub(t.get(M), t.mul(Yb, false, Au, false));
      __syncthreads();
      t.put(M, m);
      __syncthreads();
    }
    ok = gj_inverse(M, t, piv, &s_dinv, &s_p, &s_sing) && ok;   // M <- g_i
    store_blk(a.gR.at(u, i), t.get(M), t);
    for (int x = 0; x < a.nk; ++x) {
      load_blk(S, sigx[x] + i * step + u * bb, t);
      __syncthreads();
      zc v;
      if (i > 0) {
        v = t.mul(Al, false, K[x], false);     // A_{i,i-1} g^x_{i-1}
        t.put(T1, v);
        __syncthreads();
        v = zadd(t.mul(T1, false, Al, true), t.get(S));
        t.put(T2, v);
      } else {
        t.put(T2, t.get(S));
      }
      __syncthreads();
      v = t.mul(M, false, T2, false);
      t.put(T1, v);
      __syncthreads();
      v = t.mul(T1, false, M, true);           // g^x_i
      t.put(K[x], v);
      store_blk(outx[x].at(u, i), v, t);
      __syncthreads();
    }
    const int sw = iG; iG = iM; iM = sw;   // G <- g_i
  }
  // ---------------- backward sweep (G holds G_{i+1,i+1}, K[x] G^x_{i+1,i+1})
  for (int i = nb - 2; i >= 0; --i) {
    zc* G = buf[iG];
    zc* M = buf[iM];
    load_blk(Au, a.Au + i * step + u * bb, t);
    load_blk(Al, a.Al + i * step + u * bb, t);
    load_blk(M, a.gR.at(u, i), t);    // g_i
    load_blk(Yb, a.Y.at(u, i), t);
    __syncthreads();
    zc v = t.mul(M, false, Au, false);  // X = g_i A_{i,i+1}
    t.put(X, v);
    __syncthreads();
    v = t.mul(X, false, G, false);      // G_{i,i+1} = -X G_{i+1,i+1}
    v = zmake(-v.x, -v.y);
    t.put(Gu, v);
    if (a.Ru.p) store_blk(a.Ru.at(u, i), v, t);
    if (a.Rl.p) {
      const zc w = t.mul(G, false, Yb, false);   // G_{i+1,i} = -G_{i+1,i+1} Y_i
      store_blk(a.Rl.at(u, i), zmake(-w.x, -w.y), t);
    }
    __syncthreads();
    for (int x = 0; x < a.nk; ++x) {
      load_blk(T2, outx[x].at(u, i), t);        // g^x_i
      __syncthreads();
      v = t.mul(Al, false, T2, false);          // Z = A_{i+1,i} g^x_i
      t.put(T1, v);
      v = t.mul(K[x], false, X, true);          // P = G^x_{i+1,i+1} X^H
      t.put(P, v);
      __syncthreads();
      if (lowx[x].p) {                          // G^x_{i+1,i} = -G_{i+1,i+1} Z - P
        const zc w = zadd(t.mul(G, false, T1, false), t.get(P));
        store_blk(lowx[x].at(u, i), zmake(-w.x, -w.y), t);
      }
      v = t.mul(Gu, false, T1, false);          // W = G_{i,i+1} Z
      t.put(S, v);
      __syncthreads();
      // G^x_ii = g^x_i + X P - W + W^H
      v = zadd(t.get(T2), t.mul(X, false, P, false));
      if (t.on) v = zadd(zsub(v, S[t.r * ld + t.c]), zconj(S[t.c * ld + t.r]));
      __syncthreads();
      t.put(K[x], v);
      store_blk(outx[x].at(u, i), v, t);
      __syncthreads();
    }
    v = zsub(t.get(M), t.mul(Gu, false, Yb, false));   // G_ii = g_i - G_{i,i+1} Y_i
    __syncthreads();
    t.put(M, v);
    store_blk(a.gR.at(u, i), v, t);
    __syncthreads();
    const int sw = iG; iG = iM; iM = sw;   // G <- G_ii
  }
  if (threadIdx.x == 0 && !ok && a.status) a.status[u] = NEGF_ERR_SINGULAR;
}

}  // namespace

bool rgf_small_supported(int b, int mixed) { return b >= 1 && (b < 16 || (b == 16 && mixed == 0)); }

size_t rgf_small_smem(int b) { return sizeof(zc) * (size_t)kBufs * b * (b + 1); }

cudaError_t rgf_small_sweep(const SmallSweep& a, cudaStream_t s) {
  if (a.U <= 0) return cudaSuccess;
  if (a.b < 1 || a.b > kSmallB || a.nk < 0 || a.nk > 2) return cudaErrorInvalidValue;
  const size_t smem = rgf_small_smem(a.b);
  cudaError_t e = once_per_device(INIT_SMALL, [](int) {
    return cudaFuncSetAttribute(rgf_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)rgf_small_smem(kSmallB));
  });
  if (e != cudaSuccess) return e;
  rgf_small_kernel<<<a.U, kSmallThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace negf

// Batched complex block kernels on CUDA cores: FP64 GEMM and Gauss-Jordan
// inversion (FP64 or FP32 arithmetic).  These are the building blocks of the
// RGF recursions (every step is a product or an inverse of b x b blocks,
// batched over independent energy points, Sec. II of the paper).
#include <atomic>
#include <mutex>

#include "negf_internal.cuh"

namespace negf {

namespace {
std::mutex g_init_mutex;
std::atomic<bool> g_init_done[kMaxDevices][INIT_NSLOT];
}  // namespace

cudaError_t once_per_device(int slot, const std::function<cudaError_t(int device)>& init) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices || slot < 0 || slot >= INIT_NSLOT) return cudaErrorInvalidValue;
  if (g_init_done[dev][slot].load(std::memory_order_acquire)) return cudaSuccess;
  std::lock_guard<std::mutex> lock(g_init_mutex);
  if (g_init_done[dev][slot].load(std::memory_order_relaxed)) return cudaSuccess;
  e = init(dev);
  if (e == cudaSuccess) g_init_done[dev][slot].store(true, std::memory_order_release);
  return e;
}

// ---------------------------------------------------------------------------
// FP64 complex GEMM: D = alpha op(A) op(B) + beta C, one grid z-slice per unit.
// Output tile TM x TM, 256 threads, (TM/16)^2 outputs per thread, K chunks of 16
// staged through shared memory.  GB300 runs FP64 at ~1/60 of its FP32 rate, so
// this kernel is bound by the FP64 pipe, not by memory.
// ---------------------------------------------------------------------------
template <int TM>
__global__ void __launch_bounds__(256) zgemm_f64_kernel(GemmArgs g) {
  const int u = blockIdx.z;
  if (g.active && !g.active[u]) return;
  constexpr int KC = 16;
  constexpr int R = TM / 16;
  __shared__ zc As[KC][TM + 1];
  __shared__ zc Bs[KC][TM + 1];
  const int n = g.n;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TM;
  const zc* A = g.A.at(u);
  const zc* B = g.B.at(u);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  zc acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = zmake(0.0, 0.0);

  for (int k0 = 0; k0 < n; k0 += KC) {
    for (int idx = threadIdx.x; idx < TM * KC; idx += 256) {
      int mm, kk;
      if (g.opA == OP_N) { kk = idx % KC; mm = idx / KC; }
      else { mm = idx % TM; kk = idx / TM; }
      const int gm = m0 + mm, gk = k0 + kk;
      zc v = zmake(0.0, 0.0);
      if (gm < n && gk < n) v = (g.opA == OP_N) ? A[(size_t)gm * n + gk] : zconj(A[(size_t)gk * n + gm]);
      As[kk][mm] = v;
    }
    for (int idx = threadIdx.x; idx < TM * KC; idx += 256) {
      int nn, kk;
      if (g.opB == OP_N) { nn = idx % TM; kk = idx / TM; }
      else { kk = idx % KC; nn = idx / KC; }
      const int gn = n0 + nn, gk = k0 + kk;
      zc v = zmake(0.0, 0.0);
      if (gn < n && gk < n) v = (g.opB == OP_N) ? B[(size_t)gk * n + gn] : zconj(B[(size_t)gn * n + gk]);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < KC; ++kk) {
      zc a[R], b[R];
#pragma unroll
      for (int i = 0; i < R; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < R; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) zfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
  zc* D = g.D.at(u);
  const zc* C = g.C.p ? g.C.at(u) : nullptr;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= n) continue;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= n) continue;
      zc v = zmul(g.alpha, acc[i][j]);
      if (C) v = zadd(v, zmul(g.beta, C[(size_t)gm * n + gn]));
      D[(size_t)gm * n + gn] = v;
    }
  }
}

cudaError_t zgemm_f64(const GemmArgs& g, cudaStream_t s) {
  if (g.units <= 0 || g.n <= 0) return cudaSuccess;
  if (g.n <= 32) {
    dim3 grid((g.n + 31) / 32, (g.n + 31) / 32, g.units);
    zgemm_f64_kernel<32><<<grid, 256, 0, s>>>(g);
  } else {
    dim3 grid((g.n + 63) / 64, (g.n + 63) / 64, g.units);
    zgemm_f64_kernel<64><<<grid, 256, 0, s>>>(g);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Gauss-Jordan inversion with partial pivoting, one CTA per unit.
//   for k: p = first argmax_{r>=k} |W[r][k]|; swap rows p,k; d = W[k][k];
//          row k <- row k / d with W[k][k] := 1/d;
//          for r != k: f = W[r][k]; row r <- row r - f * row k with W[r][k] := -f/d
//   finally undo the row swaps as column swaps in reverse order.
// ---------------------------------------------------------------------------
template <typename R> struct CT;
template <> struct CT<double> { typedef double2 T; };
template <> struct CT<float> { typedef float2 T; };

template <typename R>
__device__ __forceinline__ typename CT<R>::T cmk(R a, R b) {
  typename CT<R>::T v; v.x = a; v.y = b; return v;
}

constexpr int kInvThreads = 1024;

// Work split: thread t owns column c = t mod n and rows r0, r0 + rs, ... with
// r0 = t div n, rs = kInvThreads div n (threads beyond rs * n only help with the
// copies); the pivot row value of its column stays in a register during the update.
// One warp finds the pivot; the row interchange is folded into the update (the old
// row k is staged in shared memory); three barriers per step.
template <typename R, bool SMEM>
__global__ void __launch_bounds__(kInvThreads) zinv_kernel(BMat X, BMat M, int n, const int* active,
                                                           typename CT<R>::T* scratch, int32_t* status) {
  typedef typename CT<R>::T C;
  const int u = blockIdx.x;
  if (active && !active[u]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* W;
  unsigned char* tail;
  if (SMEM) {
    W = reinterpret_cast<C*>(smem_raw);
    tail = smem_raw + sizeof(C) * (size_t)n * (n + 1);
  } else {
    W = scratch + (size_t)u * n * (n + 1);
    tail = smem_raw;
  }
  C* prow = reinterpret_cast<C*>(tail);
  C* fcol = prow + n;
  C* krow = fcol + n;
  int* piv = reinterpret_cast<int*>(krow + n);
  __shared__ int s_p;
  __shared__ int s_sing;
  __shared__ C s_dinv;

  const int tid = threadIdx.x, lane = tid & 31;
  const zc* Min = M.at(u);
  const int nn = n * n;
  const int ld = n + 1;   // padded row stride: column reads hit distinct banks
  for (int i = tid; i < nn; i += kInvThreads) {
    const int r = i / n, c = i - r * n;
    const zc v = Min[i];
    W[(size_t)r * ld + c] = cmk<R>((R)v.x, (R)v.y);
  }
  if (tid == 0) s_sing = 0;
  const int rs = kInvThreads / n;           // >= 1 for n <= kInvThreads
  const int mc = tid % n, r0 = tid / n;     // this thread's column and first row
  const bool upd = r0 < rs;
  __syncthreads();

  for (int k = 0; k < n; ++k) {
    // -- pivot (warp 0): first row r >= k with the largest |W[r][k]|^2
    if (tid < 32) {
      R best = (R)-1;
      int bi = n;
      for (int r = k + lane; r < n; r += 32) {
        const C v = W[(size_t)r * ld + k];
        const R a = v.x * v.x + v.y * v.y;
        if (a > best) { best = a; bi = r; }
      }
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        const R ob = __shfl_down_sync(0xffffffffu, best, off);
        const int oi = __shfl_down_sync(0xffffffffu, bi, off);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (lane == 0) {
        if (!(best > (R)0)) { s_sing = 1; bi = k; }
        s_p = bi;
        piv[k] = bi;
        const C d = W[(size_t)bi * ld + k];
        const R den = d.x * d.x + d.y * d.y;
        s_dinv = (den > (R)0) ? cmk<R>(d.x / den, -d.y / den) : cmk<R>((R)0, (R)0);
      }
    }
    __syncthreads();
    const int p = s_p;
    // -- scaled pivot row (from row p), elimination factors of the swapped rows, and a
    //    copy of the old row k (which becomes row p)
    if (tid < n) {
      const C dinv = s_dinv;
      const C v = (tid == k) ? cmk<R>((R)1, (R)0) : W[(size_t)p * ld + tid];
      prow[tid] = cmk<R>(v.x * dinv.x - v.y * dinv.y, v.x * dinv.y + v.y * dinv.x);
      fcol[tid] = (tid == k) ? cmk<R>((R)0, (R)0) : W[(size_t)(tid == p ? k : tid) * ld + k];
      krow[tid] = W[(size_t)k * ld + tid];
    }
    __syncthreads();
    // -- rank-1 update: row k <- pivot row; row r <- (swapped) row r - f_r * pivot row,
    //    the pivot column entering as 0 (so that it becomes -f_r / d)
    if (upd) {
      const C pc = prow[mc];
      const C zero = cmk<R>((R)0, (R)0);
      const C kr = krow[mc];
      int r = r0;
      // four rows per iteration: their loads are independent and issued together (FP32
      // and n >= 96, where it measured faster; the FP64 matrix of b = 128 lives in
      // global scratch, and small blocks have few rows per thread)
      if (sizeof(R) == 4 && n >= 96)
      for (; r + 3 * rs < n; r += 4 * rs) {
        C w[4], f[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int rq = r + q * rs;
          w[q] = (mc == k) ? zero : ((rq == p) ? kr : W[(size_t)rq * ld + mc]);
          f[q] = fcol[rq];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int rq = r + q * rs;
          C x = w[q];
          x.x = x.x - (f[q].x * pc.x - f[q].y * pc.y);
          x.y = x.y - (f[q].x * pc.y + f[q].y * pc.x);
          W[(size_t)rq * ld + mc] = (rq == k) ? pc : x;
        }
      }
      for (; r < n; r += rs) {
        const size_t i = (size_t)r * ld + mc;
        if (r == k) {
          W[i] = pc;
        } else {
          C w = (mc == k) ? zero : ((r == p) ? kr : W[i]);
          const C f = fcol[r];
          w.x = w.x - (f.x * pc.x - f.y * pc.y);
          w.y = w.y - (f.x * pc.y + f.y * pc.x);
          W[i] = w;
        }
      }
    }
    __syncthreads();
  }
  // -- undo the row interchanges: swap columns k and piv[k], last pivot first
  for (int k = n - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k) {
      for (int r = tid; r < n; r += kInvThreads) {
        C t = W[(size_t)r * ld + k];
        W[(size_t)r * ld + k] = W[(size_t)r * ld + p];
        W[(size_t)r * ld + p] = t;
      }
    }
    __syncthreads();
  }
  zc* Xo = X.at(u);
  for (int i = tid; i < nn; i += kInvThreads) {
    const int r = i / n, c = i - r * n;
    const C v = W[(size_t)r * ld + c];
    Xo[i] = zmake((double)v.x, (double)v.y);
  }
  if (tid == 0 && s_sing && status) status[u] = NEGF_ERR_SINGULAR;
}

// ---------------------------------------------------------------------------
// The same Gauss-Jordan inversion in panels of kPW columns.  The panel's pivot steps are
// first applied to the panel's own columns only (pivot search, row interchange, scaling
// and elimination exactly as above), recording the multiplier f_r of every row at each
// step in F (F[k][j] = d_j on the pivot row).  The other columns then take the panel's
// steps in one pass: with a column's rows permuted by the panel's interchanges into y,
// the pivot rows' new values are v_j = (y_{k0+j} - sum_{j'<j} F[k0+j][j'] v_j') / d_j,
// and row r becomes y_r - sum_j F[r][j] v_j, except pivot row k0+j, which becomes
// v_j - sum_{j'>j} F[k0+j][j'] v_j'.  The same pivots and arithmetic up to rounding
// order, with one pass over the matrix per panel instead of one per pivot step.
// ---------------------------------------------------------------------------
constexpr int kPW = 8;
constexpr int kPanelThreads = 128;   // the panel's rows, one per thread (n <= 128)

// a barrier of the first kPanelThreads threads only (the rest of the CTA waits at the
// next full barrier)
__device__ __forceinline__ void panel_barrier() { asm volatile("bar.sync 1, %0;" ::"n"(kPanelThreads) : "memory"); }

template <typename R>
static size_t panel_smem_bytes(int n) {
  typedef typename CT<R>::T C;
  return sizeof(C) * ((size_t)n * (n + 1) + 4 * (size_t)kPW * n) + 3 * sizeof(int) * (size_t)n + 16;
}

template <typename R>
__device__ __forceinline__ typename CT<R>::T cmul(typename CT<R>::T a, typename CT<R>::T b) {
  return cmk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// the kPW multipliers of one row (16-byte loads: the row starts on a 16-byte boundary)
template <typename R>
__device__ __forceinline__ void load_row(typename CT<R>::T* f, const typename CT<R>::T* src) {
  if (sizeof(typename CT<R>::T) == 8) {
    const float4* q = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int j = 0; j < kPW / 2; ++j) {
      const float4 t = q[j];
      f[2 * j].x = (R)t.x; f[2 * j].y = (R)t.y;
      f[2 * j + 1].x = (R)t.z; f[2 * j + 1].y = (R)t.w;
    }
  } else {
#pragma unroll
    for (int j = 0; j < kPW; ++j) f[j] = src[j];
  }
}

template <typename R>
__global__ void __launch_bounds__(kInvThreads) zinv_panel_kernel(BMat X, BMat M, int n, const int* active,
                                                                 int32_t* status) {
  typedef typename CT<R>::T C;
  const int u = blockIdx.x;
  if (active && !active[u]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = n + 1;
  C* W = reinterpret_cast<C*>(smem_raw);   // n x ld
  C* F = W + (size_t)n * ld;               // [row][kPW]: multipliers of the panel's steps
  C* V = F + (size_t)n * kPW;              // [kPW][n]: new pivot-row values of the other columns
  C* Stg = V + (size_t)kPW * n;            // [2 kPW][n]: rows moved by the panel's interchanges
  int* piv = reinterpret_cast<int*>(Stg + (size_t)2 * kPW * n);
  int* rowsrc = piv + n;                   // position -> row of W it holds after the interchanges
  int* stage_of = rowsrc + n;              // position -> its slot in Stg, or -1
  __shared__ C s_dinv[kPW];
  __shared__ C s_prow[kPW];
  __shared__ R s_cbest[kPanelThreads / 32];
  __shared__ int s_cpos[kPanelThreads / 32];
  __shared__ int s_sing;
  const int tid = threadIdx.x, lane = tid & 31;
  const zc* Min = M.at(u);
  const int nn = n * n;
  for (int i = tid; i < nn; i += kInvThreads) {
    const int r = i / n, c = i - r * n;
    const zc v = Min[i];
    W[(size_t)r * ld + c] = cmk<R>((R)v.x, (R)v.y);
  }
  for (int i = tid; i < n; i += kInvThreads) {
    rowsrc[i] = i;
    stage_of[i] = -1;
  }
  if (tid == 0) s_sing = 0;
  __syncthreads();
  const C zero = cmk<R>((R)0, (R)0);
  const int rs = kInvThreads / n;          // >= kPW: n <= kInvThreads / kPW
  const int mc = tid % n, r0 = tid / n;    // the other columns' pass: column and first row

  for (int k0 = 0; k0 < n; k0 += kPW) {
    const int w = min(kPW, n - k0);
    // ---- the panel's pivot steps on its own columns, by the first kPanelThreads threads:
    //      thread r keeps row r of the panel and its multipliers in registers, and the
    //      interchanges move positions (mypos: where row r stands) instead of data; two
    //      barriers of these warps per step
    if (tid < kPanelThreads) {
      const int r = tid;
      const bool has = r < n;
      C pw[kPW];
      C* pf = Stg + r * kPW;   // row r's multipliers (the staging buffer is free until the panel ends)
      int mypos = r;
#pragma unroll
      for (int j = 0; j < kPW; ++j) pw[j] = (has && j < w) ? W[r * ld + k0 + j] : zero;
#pragma unroll
      for (int j = 0; j < kPW; ++j) {
        if (j < w) {
          const int k = k0 + j;
          // pivot: the smallest position >= k holding the largest |.|^2 of column j
          R best = (R)-1;
          int bp = n;
          if (has && mypos >= k) {
            best = pw[j].x * pw[j].x + pw[j].y * pw[j].y;
            bp = mypos;
          }
#pragma unroll
          for (int off = 16; off > 0; off >>= 1) {
            const R ob = __shfl_down_sync(0xffffffffu, best, off);
            const int oi = __shfl_down_sync(0xffffffffu, bp, off);
            if (ob > best || (ob == best && oi < bp)) { best = ob; bp = oi; }
          }
          if (lane == 0) {
            s_cbest[tid >> 5] = best;
            s_cpos[tid >> 5] = bp;
          }
          panel_barrier();
          best = s_cbest[0];
          int p = s_cpos[0];
#pragma unroll
          for (int q = 1; q < kPanelThreads / 32; ++q) {
            const R ob = s_cbest[q];
            const int oi = s_cpos[q];
            if (ob > best || (ob == best && oi < p)) { best = ob; p = oi; }
          }
          if (!(best > (R)0)) p = k;   // singular: the row at position k stays
          const bool win = has && mypos == p;
          if (win) {
            const C d = pw[j];
            const R den = d.x * d.x + d.y * d.y;
            const C dinv = (den > (R)0) ? cmk<R>(d.x / den, -d.y / den) : zero;
#pragma unroll
            for (int c = 0; c < kPW; ++c) s_prow[c] = (c == j) ? dinv : cmul<R>(pw[c], dinv);
            s_dinv[j] = dinv;
            piv[k] = p;
            if (!(best > (R)0)) s_sing = 1;
          }
          panel_barrier();
          if (has) {
            if (win) {
              pf[j] = pw[j];   // F[k][j] = d
#pragma unroll
              for (int c = 0; c < kPW; ++c) pw[c] = s_prow[c];
            } else {
              const C f = pw[j];
              pf[j] = f;
#pragma unroll
              for (int c = 0; c < kPW; ++c) {
                const C pc = s_prow[c];
                if (c == j) {
                  pw[c] = cmk<R>(-(f.x * pc.x - f.y * pc.y), -(f.x * pc.y + f.y * pc.x));
                } else {
                  pw[c].x -= f.x * pc.x - f.y * pc.y;
                  pw[c].y -= f.x * pc.y + f.y * pc.x;
                }
              }
            }
            if (mypos == k) mypos = p;   // the row at position k takes the pivot row's place
            if (win) mypos = k;
          }
        }
      }
      // the panel's columns and multipliers at the rows' final positions
      if (has) {
#pragma unroll
        for (int j = 0; j < kPW; ++j) {
          if (j < w) {
            W[mypos * ld + k0 + j] = pw[j];
            F[mypos * kPW + j] = pf[j];   // this thread's own entries
          }
        }
        rowsrc[mypos] = r;
      }
    }
    __syncthreads();
    // ---- stage the rows that the interchanges moved (positions k0 .. k0+w-1 and the
    //      pivot rows' old positions; a position listed twice holds the same row in both
    //      slots) and the other columns' new pivot-row values
    if (tid < 2 * w) stage_of[tid < w ? k0 + tid : piv[k0 + tid - w]] = tid;
    for (int i = tid; i < 2 * w * n; i += kInvThreads) {
      const int sl = i / n, c = i - sl * n;
      const int pos = sl < w ? k0 + sl : piv[k0 + sl - w];
      Stg[(size_t)sl * n + c] = W[(size_t)rowsrc[pos] * ld + c];
    }
    if (tid < n && (tid < k0 || tid >= k0 + w)) {
      C v[kPW];
#pragma unroll
      for (int j = 0; j < kPW; ++j) {
        if (j < w) {
          C a = W[(size_t)rowsrc[k0 + j] * ld + tid];
#pragma unroll
          for (int q = 0; q < kPW; ++q) {
            if (q < j) {
              const C f = F[(size_t)(k0 + j) * kPW + q];
              a.x -= f.x * v[q].x - f.y * v[q].y;
              a.y -= f.x * v[q].y + f.y * v[q].x;
            }
          }
          v[j] = cmul<R>(a, s_dinv[j]);
          V[(size_t)j * n + tid] = v[j];
        }
      }
    }
    __syncthreads();
    // ---- the other columns take the panel's steps in one pass
    if (r0 < rs && (mc < k0 || mc >= k0 + w) && w == kPW) {
      // a full panel: the rows other than the pivot rows with no per-step guards (a warp
      // shares its row, so the pivot-row and moved-row branches are uniform), then this
      // thread's pivot rows
      C v[kPW];
#pragma unroll
      for (int j = 0; j < kPW; ++j) v[j] = V[j * n + mc];
      C* wp = W + r0 * ld + mc;
      const C* fp = F + r0 * kPW;
      for (int r = r0; r < n; r += rs, wp += rs * ld, fp += rs * kPW) {
        if (r >= k0 && r < k0 + kPW) continue;
        const int sl = stage_of[r];
        C a = (sl >= 0) ? Stg[sl * n + mc] : *wp;
        C f[kPW];
        load_row<R>(f, fp);
#pragma unroll
        for (int j = 0; j < kPW; ++j) {
          a.x -= f[j].x * v[j].x - f[j].y * v[j].y;
          a.y -= f[j].x * v[j].y + f[j].y * v[j].x;
        }
        *wp = a;
      }
      for (int r = k0 + ((r0 - k0) % rs + rs) % rs; r < k0 + kPW; r += rs) {
        const int jr = r - k0;
        C f[kPW];
        load_row<R>(f, F + r * kPW);
        C a = zero;
#pragma unroll
        for (int j = 0; j < kPW; ++j) {
          if (j == jr) a = v[j];
          if (j > jr) {
            a.x -= f[j].x * v[j].x - f[j].y * v[j].y;
            a.y -= f[j].x * v[j].y + f[j].y * v[j].x;
          }
        }
        W[r * ld + mc] = a;
      }
    } else if (r0 < rs && (mc < k0 || mc >= k0 + w)) {
      C v[kPW];
#pragma unroll
      for (int j = 0; j < kPW; ++j) v[j] = (j < w) ? V[(size_t)j * n + mc] : zero;
      for (int r = r0; r < n; r += rs) {
        const bool pivot_row = r >= k0 && r < k0 + w;
        const int jr = r - k0;
        C a;
        if (pivot_row) {
          a = zero;
#pragma unroll
          for (int j = 0; j < kPW; ++j)
            if (j == jr) a = v[j];
        } else {
          const int sl = stage_of[r];
          a = (sl >= 0) ? Stg[(size_t)sl * n + mc] : W[(size_t)r * ld + mc];
        }
#pragma unroll
        for (int j = 0; j < kPW; ++j) {
          if (j < w && (!pivot_row || j > jr)) {
            const C f = F[(size_t)r * kPW + j];
            a.x -= f.x * v[j].x - f.y * v[j].y;
            a.y -= f.x * v[j].y + f.y * v[j].x;
          }
        }
        W[(size_t)r * ld + mc] = a;
      }
    }
    __syncthreads();
    // the matrix is in the panel's row order now: the next panel starts from the identity
    // map (only the moved positions differ from it)
    if (tid < 2 * w) {
      const int pos = tid < w ? k0 + tid : piv[k0 + tid - w];
      stage_of[pos] = -1;
      rowsrc[pos] = pos;
    }
    // (the next panel's first barrier orders this before its staging)
  }
  // -- undo the row interchanges: swap columns k and piv[k], last pivot first
  for (int k = n - 1; k >= 0; --k) {
    const int p = piv[k];
    if (p != k) {
      for (int r = tid; r < n; r += kInvThreads) {
        C t = W[(size_t)r * ld + k];
        W[(size_t)r * ld + k] = W[(size_t)r * ld + p];
        W[(size_t)r * ld + p] = t;
      }
    }
    __syncthreads();
  }
  zc* Xo = X.at(u);
  for (int i = tid; i < nn; i += kInvThreads) {
    const int r = i / n, c = i - r * n;
    const C v = W[(size_t)r * ld + c];
    Xo[i] = zmake((double)v.x, (double)v.y);
  }
  if (tid == 0 && s_sing && status) status[u] = NEGF_ERR_SINGULAR;
}

static size_t inv_tail_bytes(int n, size_t csz) { return 3 * csz * n + sizeof(int) * n + 16; }
static const size_t kInvSmemMax = 200 * 1024;
static const size_t kPanelSmemMax = 227 * 1024;

size_t zinv_scratch_bytes(int n, int units, int single) {
  const size_t csz = single ? sizeof(float2) : sizeof(double2);
  if (csz * (size_t)n * (n + 1) + inv_tail_bytes(n, csz) <= kInvSmemMax) return 0;
  return csz * (size_t)n * (n + 1) * units;
}

template <typename R>
static cudaError_t launch_inv(BMat X, BMat M, int n, int units, const int* active, void* scratch,
                              int32_t* status, cudaStream_t s) {
  typedef typename CT<R>::T C;
  const size_t full = sizeof(C) * (size_t)n * (n + 1) + inv_tail_bytes(n, sizeof(C));
  const size_t pbytes = panel_smem_bytes<R>(n);
  // panels for the FP32 inverse (the FP64 instance would spill its panel values)
  if (sizeof(R) == 4 && n >= 16 && n <= kPanelThreads && pbytes <= kPanelSmemMax) {
    cudaError_t e = cudaFuncSetAttribute(zinv_panel_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pbytes);
    if (e != cudaSuccess) return e;
    zinv_panel_kernel<R><<<units, kInvThreads, pbytes, s>>>(X, M, n, active, status);
  } else if (full <= kInvSmemMax) {
    cudaError_t e = cudaFuncSetAttribute(zinv_kernel<R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)full);
    if (e != cudaSuccess) return e;
    zinv_kernel<R, true><<<units, kInvThreads, full, s>>>(X, M, n, active, nullptr, status);
  } else {
    if (!scratch) return cudaErrorInvalidValue;
    const size_t t = inv_tail_bytes(n, sizeof(C));
    zinv_kernel<R, false><<<units, kInvThreads, t, s>>>(X, M, n, active, (C*)scratch, status);
  }
  return cudaGetLastError();
}

cudaError_t zinv(BMat X, BMat M, int n, int units, const int* active, int single, void* scratch,
                 int32_t* status, cudaStream_t s) {
  if (units <= 0 || n <= 0) return cudaSuccess;
  if (single) return launch_inv<float>(X, M, n, units, active, scratch, status, s);
  return launch_inv<double>(X, M, n, units, active, scratch, status, s);
}

}  // namespace negf

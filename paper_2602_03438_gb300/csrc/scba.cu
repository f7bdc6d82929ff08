// Eq. (3) of the paper on a uniform energy grid, and the mixing step of the
// self-consistent scattering loop (Fig. 2):
//
//   Y[n] = sum_{m=-M..M} w_m X[n - m]     for every matrix element, X = 0 off the grid,
//
// evaluated as a zero-padded circular convolution by FFT (Sec. II: "performed more
// efficiently ... after a fast Fourier transform").  The energy axis of the Green's
// function blocks is strided (energy-major storage [e][element]): a CTA loads TE
// consecutive elements for all energies (coalesced rows of TE complex numbers), runs TE
// length-N transforms in shared memory (radix 2: decimation in time forward from
// bit-reversed positions, decimation in frequency backward into bit-reversed
// positions, so that no separate permutation pass is needed), multiplies by the
// kernel's spectrum and writes the ne convolved values back.  FP64 throughout.
#include <algorithm>

#include "negf_internal.cuh"

namespace negf {

namespace {

__device__ __forceinline__ unsigned bitrev(unsigned x, int logn) { return __brev(x) >> (32 - logn); }

__device__ __forceinline__ zc cmul(zc a, zc b) { return zmake(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }

// spectrum of the wrapped kernel: Wh[k] = sum_m w_m exp(-2 pi i k m / N)
__global__ void kernel_spectrum_kernel(const double* w, int M, int N, zc* Wh) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= N) return;
  double re = 0.0, im = 0.0;
  for (int m = -M; m <= M; ++m) {
    const double c = w[m + M];
    if (c == 0.0) continue;
    // angle -2 k m / N in units of pi, reduced to (-1, 1] exactly with integer arithmetic
    long long q = (long long)k * m % N;   // in (-N, N)
    double sn, cs;
    sincospi(-2.0 * (double)q / (double)N, &sn, &cs);
    re += c * cs;
    im += c * sn;
  }
  Wh[k] = zmake(re, im);
}

// one CTA: TE elements (columns) x N energies (rows) in shared memory
__global__ void __launch_bounds__(256) energy_conv_kernel(const zc* __restrict__ X, zc* __restrict__ Y, long long ld,
                                                          int nelem, int ne, int logn, int TE, const zc* __restrict__ Wh) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = 1 << logn;
  zc* a = reinterpret_cast<zc*>(smem_raw);      // [TE][N]
  zc* tw = a + (size_t)TE * N;                  // [N / 2]: exp(-2 pi i k / N)
  const int e0 = blockIdx.x * TE;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int k = tid; k < N / 2; k += nt) {
    double sn, cs;
    sincospi(-2.0 * (double)k / (double)N, &sn, &cs);
    tw[k] = zmake(cs, sn);
  }
  for (int i = tid; i < TE * N; i += nt) a[i] = zmake(0.0, 0.0);
  __syncthreads();
  // load into bit-reversed positions (energies beyond ne stay zero: the padding)
  for (int i = tid; i < ne * TE; i += nt) {
    const int e = i / TE, t = i - e * TE;
    if (e0 + t < nelem) a[(size_t)t * N + bitrev((unsigned)e, logn)] = X[(long long)e * ld + e0 + t];
  }
  __syncthreads();
  // forward transform, decimation in time (bit-reversed in, natural order out)
  for (int len = 2; len <= N; len <<= 1) {
    const int half = len >> 1, stride = N / len;
    for (int q = tid; q < TE * (N / 2); q += nt) {
      const int t = q / (N / 2), r = q - t * (N / 2);
      const int g = r / half, k = r - g * half;
      const int i = g * len + k, j = i + half;
      zc* col = a + (size_t)t * N;
      const zc u = col[i], v = cmul(col[j], tw[k * stride]);
      col[i] = zadd(u, v);
      col[j] = zsub(u, v);
    }
    __syncthreads();
  }
  // times the kernel's spectrum
  for (int i = tid; i < TE * N; i += nt) a[i] = cmul(a[i], Wh[i & (N - 1)]);
  __syncthreads();
  // inverse transform, decimation in frequency (natural order in, bit-reversed out),
  // conjugate twiddles
  for (int len = N; len >= 2; len >>= 1) {
    const int half = len >> 1, stride = N / len;
    for (int q = tid; q < TE * (N / 2); q += nt) {
      const int t = q / (N / 2), r = q - t * (N / 2);
      const int g = r / half, k = r - g * half;
      const int i = g * len + k, j = i + half;
      zc* col = a + (size_t)t * N;
      const zc u = col[i], v = col[j];
      col[i] = zadd(u, v);
      col[j] = cmul(zsub(u, v), zconj(tw[k * stride]));
    }
    __syncthreads();
  }
  const double inv_n = 1.0 / (double)N;
  for (int i = tid; i < ne * TE; i += nt) {
    const int e = i / TE, t = i - e * TE;
    if (e0 + t < nelem) Y[(long long)e * ld + e0 + t] = zscale(a[(size_t)t * N + bitrev((unsigned)e, logn)], inv_n);
  }
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

// stats[0] = max |SLn - SL|^2, [1] = max |SGn - SG|^2, [2] = max(|SLn|, |SGn|)^2 (squared
// moduli: two FP64 operations per entry); then SL += mix (SLn - SL), SG += mix (SGn - SG),
// SR = (SG - SL) / 2
__global__ void scba_mix_kernel(zc* SL, zc* SG, zc* SR, const zc* SLn, const zc* SGn, long long n, double mix,
                                double* stats) {
  double dl = 0.0, dg = 0.0, sc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const zc l = SL[i], g = SG[i], ln = SLn[i], gn = SGn[i];
    dl = fmax(dl, zabs2(zsub(ln, l)));
    dg = fmax(dg, zabs2(zsub(gn, g)));
    sc = fmax(sc, fmax(zabs2(ln), zabs2(gn)));
    const zc l2 = zadd(l, zscale(zsub(ln, l), mix)), g2 = zadd(g, zscale(zsub(gn, g), mix));
    SL[i] = l2;
    SG[i] = g2;
    SR[i] = zscale(zsub(g2, l2), 0.5);
  }
  for (int off = 16; off > 0; off >>= 1) {
    dl = fmax(dl, __shfl_down_sync(0xffffffffu, dl, off));
    dg = fmax(dg, __shfl_down_sync(0xffffffffu, dg, off));
    sc = fmax(sc, __shfl_down_sync(0xffffffffu, sc, off));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_nonneg(&stats[0], dl);
    atomic_max_nonneg(&stats[1], dg);
    atomic_max_nonneg(&stats[2], sc);
  }
}

}  // namespace

int conv_log2_size(int ne, int M) {
  int logn = 1;
  while ((1 << logn) < ne + M) ++logn;
  return logn;
}

size_t conv_spectrum_bytes(int ne, int M) { return sizeof(zc) * ((size_t)1 << conv_log2_size(ne, M)); }

cudaError_t energy_convolution(const zc* X, zc* Y, long long ld, int nelem, int ne, int M, const double* w_dev,
                               zc* Wh, cudaStream_t s) {
  if (ne <= 0 || nelem <= 0) return cudaSuccess;
  const int logn = conv_log2_size(ne, M);
  const int N = 1 << logn;
  if (logn > 13) return cudaErrorInvalidValue;   // N <= 8192: one column fits shared memory
  kernel_spectrum_kernel<<<(N + 255) / 256, 256, 0, s>>>(w_dev, M, N, Wh);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int TE = std::max(1, std::min(8, 8192 / N));
  const size_t smem = sizeof(zc) * ((size_t)TE * N + N / 2);
  e = cudaFuncSetAttribute(energy_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  energy_conv_kernel<<<(nelem + TE - 1) / TE, 256, smem, s>>>(X, Y, ld, nelem, ne, logn, TE, Wh);
  return cudaGetLastError();
}

cudaError_t scba_mix(zc* SL, zc* SG, zc* SR, const zc* SLn, const zc* SGn, long long n, double mix, double* stats,
                     cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(stats, 0, 3 * sizeof(double), s);
  if (e != cudaSuccess || n <= 0) return e;
  const int blocks = (int)std::min<long long>((n + 255) / 256, 4096);
  scba_mix_kernel<<<blocks, 256, 0, s>>>(SL, SG, SR, SLn, SGn, n, mix, stats);
  return cudaGetLastError();
}

}  // namespace negf

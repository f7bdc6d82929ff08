/*
 * negf.h -- C ABI of the GB300 (sm_103a) batched RGF library (libnegf.so).
 *
 * The library computes, for many energy points at once, the selected blocks of
 * the retarded and lesser Green's functions of a block-tridiagonal (BT) system
 * (paper Sec. II and Eqs. (1)-(2)):
 *
 *     G^R(E) = (z S - H - Sigma^R_L - Sigma^R_R - Sigma^R_scat)^{-1},  z = E + i eta   (Eq. (1))
 *     G^<(E) = G^R Sigma^< G^A,  Sigma^< = Sigma^<_scat + i f_L Gamma_L + i f_R Gamma_R  (Eq. (2))
 *
 * returning only the blocks on the BT pattern (Sec. II: "only selected entries
 * of C are needed"), the lead (open boundary) self-energies, and the
 * transmission, DOS, interface current and density that follow from them.
 * Every energy is independent (Sec. II); energies are the batch axis.
 *
 * Conventions (all calls):
 *  - Complex matrices are interleaved (re, im) double precision, row-major,
 *    layout-compatible with contiguous torch.complex128 / numpy complex128.
 *  - "device" means GPU global memory.  Every pointer is a device pointer
 *    owned by the caller unless the comment says "host".  The library owns
 *    only the workspace of its context.
 *  - All compute calls are asynchronous on the given CUDA stream (0 = legacy
 *    default stream).  A negative return means that nothing was enqueued
 *    (argument error) or that a launch failed; the message is available from
 *    negf_last_error().  Numerical trouble (no convergence, a singular block)
 *    is reported per energy in the caller's `status` array (device int32),
 *    and as the worst code by negf_ctx_sync().
 *  - Several independent BT devices ("ndev" > 1, the uneven batch) are packed
 *    device after device.  Offsets are exclusive prefix sums computed by the
 *    library; negf_layout() returns them so callers can address the packing.
 *
 * Per-device packing (b = bs[d], nb = nb[d], ne = ne[d]):
 *    H_diag, S_diag       : nb     blocks b x b             (device order)
 *    H_up,   S_up         : nb-1   blocks, block (i, i+1);  block (i+1, i) = (block (i,i+1))^H
 *    energy, f_L, f_R     : ne     doubles
 *    sigma_L, sigma_R     : ne     blocks (lead self-energy on block 0 / block nb-1)
 *    GR_diag, GL_diag     : ne*nb  blocks, energy-major: [e][i]
 *    GR_up, GR_low, GL_low: ne*(nb-1) blocks, [e][i]: (i,i+1), (i+1,i), (i+1,i)
 *    current              : ne*(nb-1) doubles,  density: nb*b doubles
 * G^<_{i,i+1} = -(G^<_{i+1,i})^H is not stored.
 */
#ifndef NEGF_H
#define NEGF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct negf_ctx negf_ctx;
typedef void* negf_stream;   /* a cudaStream_t */

typedef enum {
  NEGF_OK = 0,
  NEGF_ERR_ARG = -1,       /* invalid argument; nothing enqueued                     */
  NEGF_ERR_CUDA = -2,      /* a CUDA runtime call or launch failed                    */
  NEGF_ERR_NOMEM = -3,     /* workspace too small for even one energy                 */
  NEGF_ERR_NOCONV = -4,    /* per energy: OBC did not reach its residual target       */
  NEGF_ERR_SINGULAR = -5,  /* per energy: an exactly zero pivot in a block inverse    */
  NEGF_ERR_TIMEOUT = -6    /* a device-side wait ran out of its iteration budget      */
} negf_status;

typedef enum {
  NEGF_FP64 = 0,       /* every product, inverse and reduction in FP64                      */
  NEGF_MIXED = 1,      /* block products on the BF16 tensor cores with exact FP32
                          accumulation of 7-bit digit slices (FP64-class: ~2^-55 of the
                          row/column scales with the default 8 digits, see
                          negf_sliced_digits; 16 <= b <= 512, K in exact passes of 256;
                          FP64 FMA otherwise); block inverses in FP32 + two refinement
                          steps whose residual uses the same product and whose correction
                          a 5-digit one; devices with b < 16 run their sweeps in FP64 (one
                          launch); I/O complex128                                           */
  NEGF_MIXED_TF32 = 2  /* block products as 3-term TF32 splits (hi*hi + hi*lo + lo*hi) on
                          the tensor cores, FP32 accumulate in TMEM (~1e-6 relative per
                          128-wide product); inverses FP32 + refinement with an FP64
                          residual                                                          */
} negf_precision;

/* One or several independent BT devices. Host struct; device pointers inside. */
typedef struct {
  int32_t ndev;              /* number of devices (>= 1)                                 */
  const int32_t* nb;         /* host [ndev]: blocks per device (>= 1)                    */
  const int32_t* bs;         /* host [ndev]: block size (1..512)                         */
  const int32_t* ne;         /* host [ndev]: energies per device (>= 0)                  */
  const void* H_diag;        /* device, packed as above                                  */
  const void* H_up;          /* device, packed; may be NULL only if every nb == 1        */
  const void* S_diag;        /* device or NULL (S = identity)                            */
  const void* S_up;          /* device or NULL (zero off-diagonal overlap)               */
  const double* energy;      /* device [sum ne]: real part of z                          */
  double eta;                /* z = E + i*eta, eta > 0                                    */
} negf_system;

/* Block-diagonal scattering self-energies (optional; pass NULL for ballistic). */
typedef struct {
  const void* sigR;          /* retarded, or NULL                                        */
  const void* sigL;          /* lesser (anti-Hermitian), or NULL                         */
  const double* sigL_scale;  /* device [sum ne*nb] factor s[e][i] on sigL, or NULL (= 1)  */
  int32_t per_energy;        /* 0: [sum nb] blocks shared by all energies of a device;
                                1: [sum ne*nb] blocks, energy-major                        */
} negf_scattering;

/* Context: binds a CUDA device and owns `workspace_bytes` of device scratch
 * (energies are processed in chunks that fit it).  Returns NEGF_ERR_ARG for a
 * NULL out-pointer, NEGF_ERR_CUDA if the device cannot be used. */
negf_status negf_ctx_create(negf_ctx** ctx, int device, size_t workspace_bytes);
negf_status negf_ctx_destroy(negf_ctx* ctx);
/* Message of the last error raised on this context (never NULL). */
const char* negf_last_error(const negf_ctx* ctx);
/* Synchronizes `stream` and returns the worst status raised by device code since
 * the previous sync (NEGF_ERR_TIMEOUT from a device wait, NEGF_ERR_CUDA for a
 * failed kernel), then clears it. */
negf_status negf_ctx_sync(negf_ctx* ctx, negf_stream stream);

/* Host-only integer layout of a (possibly uneven) batch.  Writes, per device d,
 * 8 int64 to out[8*d .. 8*d+7]:
 *   [0] diag-block offset   (sum_{d'<d} nb*b*b)        elements into H_diag / S_diag
 *   [1] up-block offset     (sum_{d'<d} (nb-1)*b*b)    into H_up / S_up
 *   [2] energy offset       (sum_{d'<d} ne)            into energy / f / status
 *   [3] lead-block offset   (sum_{d'<d} ne*b*b)        into sigma_L / sigma_R
 *   [4] G diag offset       (sum_{d'<d} ne*nb*b*b)     into GR_diag / GL_diag
 *   [5] G off-diag offset   (sum_{d'<d} ne*(nb-1)*b*b) into GR_up / GR_low / GL_low
 *   [6] current offset      (sum_{d'<d} ne*(nb-1))     into current
 *   [7] orbital offset      (sum_{d'<d} nb*b)          into density
 * plus, at out[8*ndev .. 8*ndev+7], the totals.  `out` has 8*(ndev+1) entries. */
negf_status negf_layout(const negf_system* sys, int64_t* out);

/* Host-only work list of the batched sweeps of an uneven batch (integer work, Sec. II:
 * every energy of every device is independent).  The devices with block size `bs` and
 * ne > 0 sweep together when there are two or more of them: one launch per sweep step
 * over all their (device, energy) units, step i of the forward sweep active for the
 * units whose device has block i, step i of the backward sweep for those with block
 * i + 1.  Writes *count = the number of such units and, for each unit u in
 * device-then-energy order (each array may be NULL): unit_dev[u] (device index),
 * unit_e[u] (energy index within the device), off_d[u] = [4] + e nb b^2 and
 * off_o[u] = [5] + e (nb - 1) b^2 of negf_layout (element offsets of the unit's block 0
 * in the diagonal and the off-diagonal outputs).  Call with NULL arrays to size them. */
negf_status negf_worklist(const negf_system* sys, int32_t bs, int32_t* count, int32_t* unit_dev, int32_t* unit_e,
                          int64_t* off_d, int64_t* off_o);

/* Lead self-energies (open boundary term of B^R, Sec. II "LSE+OBC").
 * The left lead repeats block 0 with hop H_{0,1} (S likewise); the right lead
 * repeats block nb-1 with hop H_{nb-2,nb-1}.  Surface Green's functions by
 * Lopez Sancho-Rubio decimation in FP64 (stop when max|alpha|,|beta| < tol *
 * initial, at most max_iter steps), followed when needed by up to 3 FP64
 * Newton steps on the surface fixed-point equation; an energy whose surface
 * residual ||(a00 - a01 g a10) g - I||_F / sqrt(b) stays above 1e-10 gets
 * NEGF_ERR_NOCONV in status[e].  Sigma_L = a10 g_L a01, Sigma_R = a01 g_R a10.
 * prec: NEGF_FP64 runs every product in FP64; NEGF_MIXED runs the products of the
 * decimation, the residuals and the Newton steps on the digit-sliced BF16 tensor-core
 * path (FP64-class: exact FP32 accumulation of 7-bit slices, ~2^-55 of the row/column
 * scales with 8 digits) when 16 <= b <= 512, with the inverses in FP32 refined twice (twice
 * more for units whose refinement residual stays above 1e-7) and redone in FP64 for any unit
 * still above it; NEGF_MIXED_TF32 is treated as NEGF_FP64 (a TF32 product is far too coarse
 * for the 1e-10 residual).
 *
 * Warm start (optional, per lead side): with g0_L and/or g0_R given, that side
 * first takes up to 8 plain Newton steps from the guess (each step's Stein
 * equation summed by Smith doubling, at most 96 levels).  The Newton result is
 * kept when its residual is <= 1e-10 and it passes the retarded-root test: the
 * LDL^H pivots of A = i (g - g^H) all exceed -1e-12 max_k A_kk (for S = I leads
 * A is positive definite exactly for the decaying root, by the inertia theorem
 * of the Stein equation A = 2 eta g g^H + (g H01) A (g H01)^H).  Otherwise that
 * lead of that energy falls back to the decimation above, which stays the arbiter
 * of the 1e-10 residual.  The guesses have no counterpart in the paper; see
 * negf_warmstart.h for the network that produces them.
 *   g0_L, g0_R : in, device [sum ne] blocks of surface-function guesses, or NULL.
 *   sigma_L/R  : out, device [sum ne] blocks.
 *   gs_L, gs_R : out, device [sum ne] blocks: the surface functions g_L, g_R, or NULL.
 *   iters      : out, device int32 [2*sum ne]: decimation steps (L, R) per energy
 *                (0 when the warm start was kept), or NULL.
 *   newton     : out, device int32 [2*sum ne]: Newton steps (L, R) per energy, warm
 *                and polishing steps together, or NULL.
 *   status     : out, device int32 [sum ne] (NEGF_OK or a negative code), or NULL.
 * Requires nb >= 2 for every device. */
negf_status negf_obc(negf_ctx* ctx, const negf_system* sys, negf_precision prec, double tol, int32_t max_iter,
                     const void* g0_L, const void* g0_R, void* sigma_L, void* sigma_R,
                     void* gs_L, void* gs_R, int32_t* iters, int32_t* newton, int32_t* status,
                     negf_stream stream);

/* Selected blocks of G^R (Eq. (1)) by the forward/backward recursive Green's
 * function sweeps (RGF, Sec. II).  sigma_L/R from negf_obc (or any retarded
 * self-energy), scat may be NULL.  GR_diag / GR_up / GR_low: out, each may be
 * NULL (not returned).  status: device int32 [sum ne] or NULL. */
negf_status negf_rgf_retarded(negf_ctx* ctx, const negf_system* sys, negf_precision prec,
                              const void* sigma_L, const void* sigma_R,
                              const negf_scattering* scat,
                              void* GR_diag, void* GR_up, void* GR_low,
                              int32_t* status, negf_stream stream);

/* G^R and G^< = G^R Sigma^< G^A (Eq. (2)) in one fused forward/backward sweep
 * pair.  f_L, f_R: device [sum ne] lead occupations (Sigma^<_lead = i f Gamma,
 * Gamma = i (Sigma^R - Sigma^A)).  Outputs as above plus GL_diag, GL_low (each
 * may be NULL). */
negf_status negf_rgf_lesser(negf_ctx* ctx, const negf_system* sys, negf_precision prec,
                            const void* sigma_L, const void* sigma_R,
                            const double* f_L, const double* f_R,
                            const negf_scattering* scat,
                            void* GR_diag, void* GR_up, void* GR_low,
                            void* GL_diag, void* GL_low,
                            int32_t* status, negf_stream stream);

/* Selected blocks of G^R (Eq. (1)) by partitioned selected inversion (Sec. II and
 * Fig. 3: Schur complements of P partitions, a reduced system solved sequentially,
 * local reconstruction), for few energies and long devices: every step is one batched
 * launch over (energy, partition) units instead of energies alone.  Each device's nb
 * must be P L with L >= 2 (else NEGF_ERR_ARG; P = 1 is the plain recursion).  Partition
 * p eliminates blocks pL .. pL+L-2 downward, coupled to the previous partition's last
 * block; the last blocks e_p = pL+L-1 form a P-block BT system; the interiors are then
 * rebuilt from its inverse.  Work per interior block: 18 block products and 1 inverse
 * (152 b^3 real flops, against 56 b^3 for the plain recursion) for a sequential depth of
 * ~2 nb/P + 2 P steps instead of 2 nb.  Arguments as negf_rgf_retarded, with GR_diag,
 * GR_up and GR_low all required (device memory); status (device int32 [sum ne] or NULL)
 * gets the worst code of the energy's partitions.  The workspace holds ~(4 nb + 17 P)
 * blocks per energy; energies are chunked to fit it. */
negf_status negf_rgf_partitioned(negf_ctx* ctx, const negf_system* sys, negf_precision prec, int32_t P,
                                 const void* sigma_L, const void* sigma_R, const negf_scattering* scat,
                                 void* GR_diag, void* GR_up, void* GR_low, int32_t* status,
                                 negf_stream stream);

/* Selected inversion of the arrowhead BT (BTA) matrix (the block-tridiagonal-arrowhead
 * shape of the Serinv solver the paper uses): the device's A(z) of negf_rgf_retarded
 * bordered by one tip block t of size b (a gate), with overlap I on the tip and none on
 * the arrow:
 *     A_tt = z I - H_tip,   A_(t,i) = -H_(t,i),   A_(i,t) = -H_(t,i)^H,   i = 0..nb-1.
 * Every device block is eliminated downward with the tip as the boundary they all couple
 * to; the tip's Schur complement is inverted last and the blocks are rebuilt from it.
 * Work per block: 14 block products and 1 inverse (120 b^3 real flops, against 56 b^3
 * for the BT recursion).
 *   H_tip   : in, device [sum b*b]: one tip Hamiltonian per device (device after device).
 *   H_arrow : in, device [sum nb] blocks H_(t,i) (the layout of H_diag).
 *   GR_diag, GR_up, GR_low : out, the device's selected blocks of G^R (up/low required
 *             when nb > 1).
 *   G_tip   : out, device [sum ne] blocks G_tt (the layout of sigma_L).
 *   G_row, G_col : out, device [sum ne*nb] blocks G_(t,i) and G_(i,t) (the layout of GR_diag).
 * Other arguments as negf_rgf_retarded. */
negf_status negf_rgf_arrowhead(negf_ctx* ctx, const negf_system* sys, negf_precision prec, const void* H_tip,
                               const void* H_arrow, const void* sigma_L, const void* sigma_R,
                               const negf_scattering* scat, void* GR_diag, void* GR_up, void* GR_low,
                               void* G_tip, void* G_row, void* G_col, int32_t* status, negf_stream stream);

/* G^R, G^< and G^> (Eq. (2) for both B^<, B^>) in one fused sweep pair: the retarded
 * sweep once, then the lesser recursion of negf_rgf_lesser run twice, on Sigma^< and on
 *     Sigma^> = Sigma^>_scat - i (1 - f_L) Gamma_L - i (1 - f_R) Gamma_R,
 *     Sigma^>_scat = Sigma^<_scat + Sigma^R_scat - (Sigma^R_scat)^H
 * (the anti-Hermitian part of a retarded self-energy is Sigma^> - Sigma^<; for a
 * scattering struct with per-block sigL_scale, the scale applies to Sigma^<_scat only).
 * Arguments as negf_rgf_lesser, plus GG_diag ([sum ne*nb] blocks) and GG_low
 * ([sum ne*(nb-1)] blocks, (i+1, i)), each device memory or NULL; with both NULL the
 * call is negf_rgf_lesser.  G^>_{i,i+1} = -(G^>_{i+1,i})^H is not stored.  Work:
 * 56 b^3 (G^R) + 2 x 72 b^3 (G^<, G^>) real flops per block. */
negf_status negf_rgf_keldysh(negf_ctx* ctx, const negf_system* sys, negf_precision prec,
                             const void* sigma_L, const void* sigma_R,
                             const double* f_L, const double* f_R,
                             const negf_scattering* scat,
                             void* GR_diag, void* GR_up, void* GR_low,
                             void* GL_diag, void* GL_low, void* GG_diag, void* GG_low,
                             int32_t* status, negf_stream stream);

/* Eq. (3) on a uniform energy grid with a scalar kernel (M_1 = M_2 = I, C_2 a scalar
 * function of the energy transfer):
 *     Y[e][i] = sum_{m=-M..M} w[m+M] X[e-m][i],   i < nelem, X = 0 outside 0 <= e < ne,
 * for complex128 X, Y (device) with element i of energy e at X + e*ld + i (ld >= nelem).
 * w: host [2M+1].  Evaluated as a zero-padded circular convolution by FFT of size
 * N = 2^k >= ne + M (Sec. II: the energy convolution in the time domain after an FFT),
 * FP64; ne + M <= 8192 (else NEGF_ERR_ARG).  X and Y must not overlap. */
negf_status negf_energy_convolution(negf_ctx* ctx, int32_t ne, int64_t nelem, int64_t ld, int32_t M,
                                    const double* w, const void* X, void* Y, negf_stream stream);

/* Scalar boson kernel of the scattering self-energies (the C_2 of Eq. (3)). */
typedef struct {
  int32_t M;                 /* support: energy transfers m dE, m = -M..M (dE: the grid step) */
  const double* w_lesser;    /* host [2M+1]: Sigma^<(E) += w_lesser[m+M] G^<(E - m dE)       */
  const double* w_greater;   /* host [2M+1]: Sigma^>(E) += w_greater[m+M] G^>(E - m dE)      */
} negf_boson_kernel;

/* The self-consistent scattering loop of Fig. 2 (the Born approximation with a scalar
 * boson kernel), on the diagonal blocks:
 *   repeat: G^R, G^<, G^> of all energies (negf_rgf_keldysh) with the current
 *           block-diagonal Sigma^R_scat, Sigma^<_scat (per energy);
 *           Sigma^x_new(E) = sum_m w^x_m G^x_ii(E - m dE) for x = <, > (Eq. (3), by FFT);
 *           change = max(max|Sigma^<_new - Sigma^<|, max|Sigma^>_new - Sigma^>|)
 *                    / max(|Sigma^<_new|, |Sigma^>_new|);
 *           Sigma^x += mixing (Sigma^x_new - Sigma^x);  Sigma^R = (Sigma^> - Sigma^<) / 2
 *           (the anti-Hermitian part; no principal-value part);
 *   until change < tol or max_iter sweeps.
 * Every device's energies must be a uniform grid whose step dE is the kernel's; the
 * returned G blocks are those of the last sweep (made with the Sigma before its update).
 *   sigR_scat, sigL_scat, sigG_scat: in/out, device [sum ne*nb] blocks (energy-major,
 *     the per_energy layout of negf_scattering): start values (zero for a cold start),
 *     then the mixed self-energies.
 *   GR_diag, GL_diag, GG_diag required; GR_up, GR_low, GL_low, GG_low may be NULL.
 *   iters, change: host out (sweeps done, last change), each may be NULL.
 * The workspace must also hold 2 [sum ne*nb] blocks for the new self-energies (else
 * NEGF_ERR_NOMEM).  The host reads the change after every sweep (one synchronization
 * per sweep). */
negf_status negf_scba(negf_ctx* ctx, const negf_system* sys, negf_precision prec,
                      const void* sigma_L, const void* sigma_R, const double* f_L, const double* f_R,
                      const negf_boson_kernel* kern, double mixing, double tol, int32_t max_iter,
                      void* sigR_scat, void* sigL_scat, void* sigG_scat,
                      void* GR_diag, void* GR_up, void* GR_low, void* GL_diag, void* GL_low,
                      void* GG_diag, void* GG_low, int32_t* status, int32_t* iters, double* change,
                      negf_stream stream);

/* The sweeps and the observables of every energy without storing any Green's function
 * block for the caller: energies are processed in chunks that fit the workspace, each
 * chunk's G^R and G^< blocks kept there only until its observables (as negf_observables)
 * are taken.  For batches whose blocks do not fit the GPU's memory (a b = 512, nb = 32
 * device needs 628 MB of blocks per energy).  Arguments as negf_rgf_lesser and
 * negf_observables (prec applies to both); T, dos, current, density may each be NULL;
 * density accumulates over all chunks with the weights e_weight. */
negf_status negf_rgf_observables(negf_ctx* ctx, const negf_system* sys, negf_precision prec,
                                 const void* sigma_L, const void* sigma_R, const double* f_L, const double* f_R,
                                 const negf_scattering* scat, const double* e_weight,
                                 double* T, double* dos, double* current, double* density,
                                 int32_t* status, negf_stream stream);

/* Observables (Sec. III: DOS, spectral current, current conservation), traces and sums
 * in FP64.  prec: the two block products of T (Gamma_L G_00 and G_00 Gamma_L) run in FP64
 * with NEGF_FP64 and NEGF_MIXED_TF32, on the digit-sliced tensor-core path (FP64-class,
 * 16 <= b <= 512) with NEGF_MIXED; any other value is NEGF_ERR_ARG.
 *   T[e]      = Tr[Gamma_L i(G_00 - G_00^H)] - Tr[Gamma_L G_00 Gamma_L G_00^H]     (needs GR_diag)
 *   dos[e]    = -(1/pi) Im Tr[G^R S] over the BT pattern                          (needs GR_diag,
 *               and GR_up, GR_low when S_up != NULL)
 *   current[e][i] = 2 Re Tr[(H_{i,i+1} - z S_{i,i+1}) G^<_{i+1,i}]                 (needs GL_low)
 *   density[k] = sum_e w[e] Re(-i (G^< S)_kk) / (2 pi)                          (needs GL_diag,
 *               GL_low when S_up != NULL; e_weight device [sum ne])
 * Each output may be NULL (skipped).  T: [sum ne], dos: [sum ne]. */
negf_status negf_observables(negf_ctx* ctx, const negf_system* sys, negf_precision prec,
                             const void* sigma_L, const double* e_weight,
                             const void* GR_diag, const void* GR_up, const void* GR_low,
                             const void* GL_diag, const void* GL_low,
                             double* T, double* dos, double* current, double* density,
                             negf_stream stream);

/* Building blocks of the sweeps, exposed for testing and reuse.
 *
 * Batched complex block product (every step of the RGF recursions is one):
 *   D[u] = alpha op_A(A[u]) op_B(B[u]) + beta C[u],  u = 0..units-1, n x n row-major
 * complex128 blocks; X[u] lives at X + u * x_stride (elements; 0 = one block shared
 * by all units).  op: 0 = as stored, 2 = conjugate transpose.  alpha, beta: host
 * double[2] (re, im).  C may be NULL (beta ignored) or equal to D; D must not
 * overlap A or B.  NEGF_FP64: FP64 FMA; NEGF_MIXED: digit-sliced BF16 tensor-core
 * product for 16 <= n <= 512 (K in exact passes of 256); NEGF_MIXED_TF32: 3-term TF32 split for n >= 16
 * (FP64 FMA outside those ranges). */
negf_status negf_block_gemm(negf_ctx* ctx, negf_precision prec, int32_t n, int32_t units, int32_t opA,
                            int32_t opB, const double* alpha, const void* A, int64_t a_stride, const void* B,
                            int64_t b_stride, const double* beta, const void* C, int64_t c_stride, void* D,
                            int64_t d_stride, negf_stream stream);
/* Batched block inverse X[u] = M[u]^{-1} (unit stride n*n; X may equal M):
 * Gauss-Jordan with partial pivoting (first largest |.| in row order).
 * NEGF_FP64: in FP64.  NEGF_MIXED / NEGF_MIXED_TF32: in FP32, then two / one
 * refinement steps X <- X + X (I - M X) with the residual formed with FP64-class
 * accuracy (the sliced tensor-core product, or FP64 FMA).  status (device
 * int32 [units] or NULL) gets NEGF_ERR_SINGULAR on an exactly zero pivot. */
negf_status negf_block_inverse(negf_ctx* ctx, negf_precision prec, int32_t n, int32_t units, const void* M,
                               void* X, int32_t* status, negf_stream stream);

/* No-allocation variant of negf_block_gemm with NEGF_MIXED precision.
 *
 * No counterpart in the paper: this is a service for callers that cannot allocate
 * device memory -- an application that owns all device memory through its own
 * arena and forbids libraries to allocate, or a latency-critical loop that cannot
 * afford the device synchronization of cudaMalloc / cudaFree.  Such callers cannot
 * create a negf_ctx (whose workspace is allocated), so this call takes no context
 * and allocates nothing.  The caller passes every input and output, with the same
 * meaning and layout as negf_block_gemm; `stream` is any stream of the current
 * device.
 *
 * The only scratch, the per-row / per-column scale exponents of the sliced product
 * (4 bytes x 2 n per unit, for 16 <= n <= 256), lives in a static device array of
 * NEGF_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until the
 * process exits.  Calls with 2 n units x 4 bytes above that size are rejected with
 * NEGF_ERR_ARG and a message from negf_last_error(NULL); split the batch.  Other n
 * use FP64 FMA and no scratch.  Every call looks up the array's device address on the
 * current device (cudaGetSymbolAddress: host-side, allocates nothing), so the call
 * stays valid across cudaDeviceReset, after which the array is loaded afresh (its old
 * contents are gone, which this call never relies on); the first call on a device may
 * load the library's device code there, so make it before any stream capture.  The
 * kernels' function attributes are set once per device.  All calls share the array and it
 * keeps the last call's contents (every scale a call reads is written by that same
 * call first, so nothing needs clearing); calls whose kernels overlap on the GPU
 * (other streams) race on it -- serialize them.  `status` (device int32 or NULL)
 * receives, through atomicMax, the magnitude of NEGF_ERR_TIMEOUT if a device-side
 * wait ran out; the caller clears it. */
#define NEGF_NOALLOC_SCRATCH_BYTES (1u << 20)
negf_status negf_block_gemm_noalloc(int32_t n, int32_t units, int32_t opA, int32_t opB, const double* alpha,
                                    const void* A, int64_t a_stride, const void* B, int64_t b_stride,
                                    const double* beta, const void* C, int64_t c_stride, void* D,
                                    int64_t d_stride, int32_t* status, negf_stream stream);

/* Autotuner of the NEGF_MIXED block products' tile shapes.  Variants:
 *   1 = half-width tiles (128 rows x 16 complex columns, two CTAs per SM; n <= 128),
 *   2 = persistent full-width tiles (128 x 32, the epilogue of one unit overlapping the
 *       next unit's MMAs; n <= 128),
 *   3 = full-width tiles, one CTA per tile (any n, K in exact passes of 256),
 *   0 = the built-in rule (1 for n <= 96, 2 for n <= 128, 3 above).
 * negf_tune_products times every variant that supports n on `units` random n x n
 * products in the context's workspace (1 warm-up + 3 calls each, CUDA events on
 * `stream`), makes the fastest the context's choice for n and returns it in *choice
 * (0 when no sliced product exists for n); ms (host [4] or NULL) gets each variant's
 * time per call (-1 where not timed).  It synchronizes the stream.  NEGF_ERR_NOMEM if
 * the workspace cannot hold 3 units x n^2 blocks and the product's scratch.
 * negf_set_product_variant sets the choice for n directly (e.g. from a saved tuning). */
negf_status negf_tune_products(negf_ctx* ctx, int32_t n, int32_t units, int32_t* choice, double* ms,
                               negf_stream stream);
negf_status negf_set_product_variant(negf_ctx* ctx, int32_t n, int32_t variant);

/* Digits per value of the NEGF_MIXED sliced product in this build (NEGF_OZ_DIGITS at
 * compile time, 6..8; 8 by default): NS digits of 7 bits give an error of ~2^(1 - 7 NS)
 * of the row x column scales and NS (NS + 1) / 2 BF16 slice-pair products per complex
 * product.  Not a paper operation: build introspection for measurement. */
int32_t negf_sliced_digits(void);

/* Kernel timing (the tracing facility).  When enabled, every launch of the
 * block-GEMM and block-inverse kernels is bracketed by CUDA events recorded on
 * the launch stream; negf_profile_read() synchronizes on those events and
 * accumulates them.  Not a paper operation: measurement support. */
negf_status negf_profile_enable(negf_ctx* ctx, int enable);
/* Accumulated since the last reset: `launches` = all kernels this context has
 * launched; per kernel class k (0 = TF32-split GEMM, 1 = FP64 GEMM, 2 = FP32
 * inverse, 3 = FP64 inverse, 4 = other (masked launches), 5 = sliced BF16 GEMM,
 * 6 = sliced BF16 GEMM with 5 digits, the refinement's correction products)
 * the launches, total milliseconds,
 * algorithmic flops (8 n^3 per complex n x n product or inverse, times the
 * units) and algorithmic bytes (16 n^2 per operand read or written).  Each
 * array has 7 entries; any pointer may be NULL. */
negf_status negf_profile_read(negf_ctx* ctx, int64_t* launches, int64_t* k_launches, double* k_ms,
                              double* k_flops, double* k_bytes);
negf_status negf_profile_reset(negf_ctx* ctx);

/* Failure-detection self test (not a paper operation).  Launches one CTA whose thread
 * waits, with the bounded device wait every tensor-core kernel of this library uses (an
 * mbarrier try_wait loop limited by %globaltimer), on an mbarrier that nothing arrives
 * on; after `wait_ns` of GPU time (1e6 <= wait_ns <= 2e9) the wait gives up and the
 * kernel raises NEGF_ERR_TIMEOUT on the context, exactly as a product kernel whose
 * operands never arrive would, and returns.  No copy, MMA or other CTA is in flight, so
 * the context stays usable; the next negf_ctx_sync(ctx, stream) returns
 * NEGF_ERR_TIMEOUT and clears it.  Returns NEGF_OK once launched, NEGF_ERR_ARG for a
 * budget out of range, NEGF_ERR_CUDA if the launch fails. */
negf_status negf_selftest_wait_timeout(negf_ctx* ctx, int64_t wait_ns, negf_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* NEGF_H */

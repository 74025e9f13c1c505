// Internal declarations shared by the CUDA translation units of libie.
// Complex arithmetic is complex128 held in double2 (x = real, y = imaginary).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <vector>

#include "../../include/ie.h"

typedef double2 cplx;

#define IE_HD __host__ __device__ __forceinline__

IE_HD cplx cmk(double re, double im) { return make_double2(re, im); }
IE_HD cplx cadd(cplx a, cplx b) { return make_double2(a.x + b.x, a.y + b.y); }
IE_HD cplx csub(cplx a, cplx b) { return make_double2(a.x - b.x, a.y - b.y); }
IE_HD cplx cscale(cplx a, double s) { return make_double2(a.x * s, a.y * s); }
IE_HD cplx cconj(cplx a) { return make_double2(a.x, -a.y); }
IE_HD cplx cmul(cplx a, cplx b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// c + a*b
IE_HD cplx cfma(cplx a, cplx b, cplx c) {
  return make_double2(fma(a.x, b.x, fma(-a.y, b.y, c.x)), fma(a.x, b.y, fma(a.y, b.x, c.y)));
}
// c - a*b
IE_HD cplx cfms(cplx a, cplx b, cplx c) {
  return make_double2(fma(-a.x, b.x, fma(a.y, b.y, c.x)), fma(-a.x, b.y, fma(-a.y, b.x, c.y)));
}
// c + conj(a)*b
IE_HD cplx cfma_conj(cplx a, cplx b, cplx c) {
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, c.x)), fma(a.x, b.y, fma(-a.y, b.x, c.y)));
}
IE_HD double cabs2(cplx a) { return fma(a.x, a.x, a.y * a.y); }
IE_HD double cabs1(cplx a) { return fabs(a.x) + fabs(a.y); }
IE_HD double cabsv(cplx a) { return hypot(a.x, a.y); }
// a / b by Smith's algorithm (R. L. Smith, CACM 5(8), 1962).
IE_HD cplx cdiv(cplx a, cplx b) {
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, d = b.x + b.y * r;
    return make_double2((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  } else {
    double r = b.x / b.y, d = b.y + b.x * r;
    return make_double2((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
}
IE_HD cplx crcp(cplx b) { return cdiv(make_double2(1.0, 0.0), b); }

// ---- status words written by kernels (device memory, one int each) ----
enum {
  ST_SINGULAR = 0,   // first zero pivot column + 1 over all poles (0 = none)
  ST_TIMEOUT = 1,    // nonzero if a bounded wait gave up
  ST_ABORT = 2,      // set to make cooperating CTAs leave early
  ST_COUNT = 8
};

#define IE_MAX_DIAG 16

// Bounded-wait limit for device spin loops, in nanoseconds of %globaltimer.
#define IE_WAIT_NS (2000ull * 1000ull * 1000ull)

__device__ __forceinline__ unsigned long long ie_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Raises a kernel's dynamic shared-memory limit to the device's per-block opt-in maximum
// (less its static shared memory). Every caller sets the same value, so launches of one kernel
// from several host threads with different sizes cannot lower the limit under one another,
// as setting the exact size before each launch would.
inline cudaError_t ie_smem_optin(const void* kfn) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, kfn);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              optin - (int)fa.sharedSizeBytes);
}

// Process-wide count of kernel launches issued by this library (exposed in ie_stats).
void ie_count_launch();
int64_t ie_launch_count();

// ---------------- kernel launchers (defined in ie_band.cu / ie_krylov.cu / ie_hsrr.cu) -------
struct DiaDev {
  int64_t n;
  int ndiag;
  int64_t off[IE_MAX_DIAG];
  const cplx* A;  // ndiag * n
  const cplx* B;
};

// Y[:, c] = (alpha_A A + alpha_B B) X[:, c] for c < k; X column c starts at X + xoff[c]
// when xoff != nullptr, else at X + c*ldx. Y column c at Y + c*ldy.
void launch_spmv(const DiaDev& P, cplx alphaA, cplx alphaB, const cplx* X, int64_t ldx,
                 const int64_t* xoff, int k, cplx* Y, int64_t ldy, cudaStream_t s);
// Assemble K_i = p_i B - A into LAPACK band storage for all q poles (columns >= n zeroed),
// in complex128 or (mixed precision) complex64.
void launch_assemble(const DiaDev& P, const cplx* d_poles, int q, int kl, int ldab,
                     int64_t n_pad, cplx* AB, cudaStream_t s);
void launch_assemble(const DiaDev& P, const cplx* d_poles, int q, int kl, int ldab,
                     int64_t n_pad, float2* AB, cudaStream_t s);
// Batched band LU with partial pivoting, all q poles in one cooperative launch.
// Ring slots per pole for the LU's published pivots (> the CTAs per pole it will use).
int band_lu_ring_slots(int q);
// sizes of the LU's publication ring for q poles: multiplier elements (of the factor type,
// allocated as complex128 they cover either precision) and int offsets
size_t band_lu_ring_elems(int q, int kl);
size_t band_lu_ring_ints(int q);
cudaError_t launch_band_lu(int q, int64_t n, int kl, int ldab, int64_t n_pad, cplx* AB,
                           int* piv, cplx* dinv, cplx* ring, int* ring_tp, unsigned* ring_flag,
                           int R, int* status, cudaStream_t s, int* ctas_per_pole);
// The same factorisation in complex64 with FP32 arithmetic (the mixed-precision path).
cudaError_t launch_band_lu(int q, int64_t n, int kl, int ldab, int64_t n_pad, float2* AB,
                           int* piv, float2* dinv, float2* ring, int* ring_tp,
                           unsigned* ring_flag, int R, int* status, cudaStream_t s,
                           int* ctas_per_pole);
// Forward (P, L) then backward (U) band solves for all q poles and k RHS columns;
// Xp[i] (n x k, ld = ldx, pole stride xstride) = w_i K_i^{-1} RHS.
// L64/U64: the split complex128 factors (launch_factors_split64); Tb/Hb/Ub: the per-panel
// block transforms of launch_block_transforms.
cudaError_t launch_band_solve(int q, int64_t n, int kl, int64_t n_pad, const cplx* L64,
                              const cplx* U64,
                              const int* piv, const cplx* dinv, const cplx* Tb, const int* Hb,
                              const cplx* Ub, const cplx* d_weights, const cplx* RHS, int64_t ldr,
                              int k, cplx* Xp, int64_t ldx, int64_t xstride, int* status,
                              cudaStream_t s);
// Batched band solves of many problems in one launch per element type. Each add_* takes the
// arguments of launch_band_solve / launch_band_solve32 for one problem; launch issues them.
struct BandSolveBatch;
BandSolveBatch* band_solve_batch_create();
void band_solve_batch_destroy(BandSolveBatch* b);
void band_solve_batch_clear(BandSolveBatch* b);
int band_solve_batch_size(const BandSolveBatch* b);
void band_solve_batch_add64(BandSolveBatch* b, int q, int64_t n, int kl, int64_t n_pad,
                            const cplx* L64, const cplx* U64, const int* piv, const cplx* dinv,
                            const cplx* Tb, const int* Hb, const cplx* Ub, const cplx* d_weights,
                            const cplx* RHS, int64_t ldr, int k, cplx* Xp, int64_t ldx,
                            int64_t xstride, int* status);
void band_solve_batch_add32(BandSolveBatch* b, int q, int64_t n, int kl, int64_t n_pad,
                            const float2* L32, int64_t ldl, const float2* U32, int64_t ldu,
                            const int* piv, const float2* dinv32, const float2* T32,
                            const int* Hb, const float2* Ui32, const cplx* d_weights,
                            const float2* RHS, int64_t ldr, int64_t rstride, int k, float2* Y32,
                            int64_t ldy, int64_t ystride, cplx* X, int64_t ldx, int64_t xstride,
                            int accumulate, int* status);
cudaError_t band_solve_batch_launch(BandSolveBatch* b, cudaStream_t s);
// Per (pole, 8-column panel): forward 16x16 transform T with its member rows H, backward
// inverse of the 8x8 diagonal block of U (complex128; complex64 copies when T32/Ui32 != null).
void launch_block_transforms(int q, int64_t n, int64_t n_pad, int kl, int ldab, const cplx* AB,
                             const int* piv, const cplx* dinv, cplx* T, int* H, cplx* Ui,
                             float2* T32, float2* Ui32, cudaStream_t s);
// The same from the complex64 band LU: complex64 T32, Ui32 (formed in FP64, rounded) and H.
void launch_block_transforms(int q, int64_t n, int64_t n_pad, int kl, int ldab, const float2* AB,
                             const int* piv, const float2* dinv, int* H, float2* T32,
                             float2* Ui32, cudaStream_t s);
// kernel family of the last tuned band-solve launch in this process (fp32 = 0: complex128,
// 1: complex64): 0 barrier-synchronised, 1 warp-specialised, 2 look-ahead; -1 none yet
int band_solve_last_kernel(int fp32);
// Mixed precision: complex64 band solves; X (FP64, per pole) = x (accumulate = 0), or
// (accumulate = 1) x is written in place over the forward result in Y32 and X is untouched.
// RHS column c of pole i at RHS + i*rstride + c*ldr (rstride 0: shared right-hand side).
cudaError_t launch_band_solve32(int q, int64_t n, int kl, int64_t n_pad, const float2* L32,
                                int64_t ldl, const float2* U32, int64_t ldu, const int* piv,
                                const float2* dinv32, const float2* T32, const int* Hb,
                                const float2* Ui32, const cplx* d_weights, const float2* RHS,
                                int64_t ldr, int64_t rstride, int k, float2* Y32, int64_t ldy,
                                int64_t ystride, cplx* X, int64_t ldx, int64_t xstride,
                                int accumulate, int* status, cudaStream_t s);
// complex128 split copy: L64 (n_pad x kl per pole), U64 (n_pad x 2kl per pole)
void launch_factors_split64(int q, int64_t n_pad, int kl, int ldab, const cplx* AB, cplx* L64,
                            cplx* U64, cudaStream_t s);
// complex64 split copy from the complex64 band LU: L32 (n_pad x klp per pole), U32 (n_pad x
// 2kl per pole) and diag32 = U(j, j) (n_pad per pole; nullable)
void launch_factors_split32(int q, int64_t n_pad, int kl, int ldab, int klp, const float2* AB,
                            float2* L32, float2* U32, float2* diag32, cudaStream_t s);
void launch_pole_residual(const DiaDev& P, const cplx* d_poles, int q, int k, const cplx* BV,
                          int64_t ldb, const cplx* X, int64_t ldx, int64_t xstride, float2* R32,
                          int64_t ldr, int64_t rstride, cudaStream_t s);
void launch_to_c64(int64_t n, int k, const cplx* X, int64_t ldx, float2* Y, int64_t ldy,
                   cudaStream_t s);
// X[i] += D[i] (FP32 correction widened to FP64) for all q poles; per (pole, column) the
// largest |.|_1 of the correction and of the new X into nrm[(i*k + c)*2 + {0,1}] as float bits
// (atomicMax; zero nrm first).
void launch_refine_add(int q, int64_t n, int k, const float2* D, int64_t ldd, int64_t dstride,
                       cplx* X, int64_t ldx, int64_t xstride, unsigned* nrm, cudaStream_t s);
// GV[:, c] = sum_i w_i Xp[i][:, c]
void launch_pole_wsum(int q, int64_t n, int k, const cplx* Xp, int64_t ldx, int64_t xstride,
                      const cplx* w, cplx* GV, int64_t ldg, cudaStream_t s);
// GV[:, c] = sum_i Xp[i][:, c]
void launch_pole_sum(int q, int64_t n, int k, const cplx* Xp, int64_t ldx, int64_t xstride,
                     cplx* GV, int64_t ldg, cudaStream_t s);
void launch_norm1_cols(const DiaDev& P, int which, double* d_out, double* d_scratch,
                       cudaStream_t s);

// ---- Krylov (ie_krylov.cu) ----
struct KrylovDev {
  int64_t n;
  int m_max;
  cplx* V;       // kmax * (m_max+1) * n ; column c basis at V + c*(m_max+1)*n
  cplx* H;       // kmax * (m_max+1) * m_max ; H_c col-major ld m_max+1
  double* beta;  // kmax
  int* jc;       // kmax : Arnoldi steps taken per column
  int* brk;      // kmax : breakdown flag
};

// Column norms of an n x k block (partial sums in scratch, result in d_out[k]).
void launch_colnorm2(int64_t n, int k, const cplx* X, int64_t ldx, double* d_out,
                     double* d_scratch, cudaStream_t s);
// Start Krylov spaces: beta_c = ||Yt_c||, V_c[:,0] = Yt_c / beta_c, jc = 0.
void launch_krylov_start(const KrylovDev& K, int k, const cplx* Yt, int64_t ldy, double* scratch,
                         cudaStream_t s);
// Offsets of V_c[:, jc[c]] for the active list (for the SpMV gather).
void launch_active_offsets(const KrylovDev& K, const int* act, int kact, int64_t* d_off,
                           cudaStream_t s);
// One Arnoldi step (CGS2) for the active columns; W (n x kact) is G applied to v_j.
void launch_arnoldi_cgs2(const KrylovDev& K, const int* act, int kact, cplx* W, int64_t ldw,
                         cplx* hbuf, double* scratch, cudaStream_t s);
// Multi-shift Givens update over H columns [jc_from, jc_to) per (column, shift);
// writes per-column max relative residual into d_res[act index].
void launch_givens(const KrylovDev& K, const int* act, int kact, const cplx* d_shifts,
                   int nshift, cplx* rot_c, cplx* rot_s, cplx* gvec, int from_zero,
                   double* d_res, cudaStream_t s);
// Final combine: U_c = V_c (sum_l wt_l y_l) + odd*beta_c v_0 for all k columns.
void launch_krylov_combine(const KrylovDev& K, int k, const cplx* d_shifts, const cplx* d_wts,
                           int nshift, double odd, cplx* Rscratch, cplx* zbuf, cplx* U,
                           int64_t ldu, cudaStream_t s);

// ---- block orthogonalisation / HSRR (ie_hsrr.cu) ----
// In-place CGS2 orthonormalisation of the n x k block Q with the rank guard;
// replaced columns get counter-based random vectors from (seed, salt, column).
void launch_orth_cgs2(int64_t n, int k, cplx* Q, int64_t ldq, uint64_t seed, uint32_t salt,
                      cplx* hbuf, double* scratch, int* flags, cudaStream_t s);
// C (k x k, col-major ld k) = W^H Y for n x k blocks.
void launch_gram(int64_t n, int k, const cplx* W, int64_t ldw, const cplx* Y, int64_t ldy,
                 cplx* C, cplx* scratch, cudaStream_t s);
// Complex QZ of (Ah, Bh) (k x k) + right eigenvectors: alpha, beta (k each),
// M = P_R V_R (k x k col-major). One CTA.
cudaError_t launch_qz(int k, cplx* Ah, cplx* Bh, cplx* Z, cplx* alpha, cplx* beta, cplx* M,
                      int* status, cudaStream_t s);
// Y (n x k) = X (n x k) * M (k x k).
void launch_gemm_small(int64_t n, int k, const cplx* X, int64_t ldx, const cplx* M, cplx* Y,
                       int64_t ldy, cudaStream_t s);
// X[:, c] /= ||X[:, c]||.
void launch_normalize_cols(int64_t n, int k, cplx* X, int64_t ldx, double* scratch,
                           cudaStream_t s);
// Residual norms per column: out[3c+0] = ||A x - lam B x||^2, out[3c+1] = ||B x||^2,
// out[3c+2] = ||x||^2.
void launch_residual_norms(const DiaDev& P, int k, const cplx* X, int64_t ldx, const cplx* lam,
                           double* d_out, double* scratch, cudaStream_t s);
// Y[:, c] = X[:, perm[c]]
void launch_permute_cols(int64_t n, int k, const cplx* X, int64_t ldx, const int* perm, cplx* Y,
                         int64_t ldy, cudaStream_t s);
// Counter-based random complex Gaussian block (SplitMix64 + Box-Muller).
void launch_random_block(int64_t n, int k, cplx* X, int64_t ldx, uint64_t seed, uint32_t salt,
                         cudaStream_t s);
// generic copies
void launch_copy_cols(int64_t n, int k, const cplx* X, int64_t ldx, cplx* Y, int64_t ldy,
                      cudaStream_t s);

// ---- adjoint pencil and sensitivities (ie_adjoint.cu) ----
// (A^H, B^H) in DIA form into AH, BH (ndiag * n each); *PH describes them.
void launch_dia_adjoint(const DiaDev& P, cplx* AH, cplx* BH, DiaDev* PH, cudaStream_t s);
// U by rows from the band LU: row j's U(j, j+1..j+2kl) at Ut + (pole*n_pad + j)*2kl.
void launch_u_rows(int q, int64_t n, int64_t n_pad, int kl, int ldab, const cplx* AB, cplx* Ut64,
                   float2* Ut32, cudaStream_t s);
void launch_u_rows(int q, int64_t n, int64_t n_pad, int kl, int ldab, const float2* AB,
                   float2* Ut32, cudaStream_t s);
// Per (pole, 8-row panel): the 16x24 transform of the conjugate-transpose L sweep on the
// members Hb (complex128 into M64; complex64 copy when M32 != null).
void launch_adj_transforms(int q, int64_t n, int64_t n_pad, int kl, int ldab, const cplx* AB,
                           const int* piv, const int* Hb, cplx* M64, float2* M32, cudaStream_t s);
void launch_adj_transforms(int q, int64_t n, int64_t n_pad, int kl, int ldab, const float2* AB,
                           const int* piv, const int* Hb, float2* M32, cudaStream_t s);
// Xp[i] = conj(w_i) K_i^{-H} RHS for all q poles (complex128 factors).
cudaError_t launch_band_solve_adj(int q, int64_t n, int kl, int64_t n_pad, const cplx* L64,
                                  const cplx* Ut64, const cplx* Ub, const cplx* M64, const int* Hb,
                                  const cplx* d_wconj, const cplx* RHS, int64_t ldr, int k,
                                  cplx* Xp, int64_t ldx, int64_t xstride, int* status,
                                  cudaStream_t s);
// complex64 factors, FP32 solve: X (FP64, per pole) = K~_i^{-H} RHS_i (accumulate = 0), or
// (accumulate = 1) the solution in place into Y32 (complex64), X untouched.
cudaError_t launch_band_solve_adj32(int q, int64_t n, int kl, int64_t n_pad, const float2* L32,
                                    int64_t ldl, const float2* Ut32, const float2* Ui32,
                                    const float2* M32, const int* Hb, const cplx* d_wconj,
                                    const float2* RHS, int64_t ldr, int64_t rstride, int k,
                                    float2* Y32, int64_t ldy, int64_t ystride, cplx* X,
                                    int64_t ldx, int64_t xstride, int accumulate, int* status,
                                    cudaStream_t s);
// den_i = y_i^H B x_i (BX: n x nf scratch); S[j, i] = alpha conj(y_i[j]) x_i[j] / den_i
// (S nullable); grad[j] = Re sum_i conj(gbar_i) S[j, i] (grad nullable; gbar device).
void launch_sensitivity(const DiaDev& P, int nf, const cplx* X, int64_t ldx, const cplx* Y,
                        int64_t ldy, cplx alpha, cplx* BX, cplx* den, cplx* S, int64_t lds,
                        const cplx* gbar, double* grad, cudaStream_t s);

// Read-only view of a handle's factorisation (defined in ie_capi.cu).
struct IeFactorsView {
  int dev;
  DiaDev P;
  int64_t n, n_pad;
  int kl, ldab, q;
  const cplx* AB;
  const cplx* L64;
  const cplx* U64;
  const int* piv;
  const cplx* dinv;
  const cplx* Tb;
  const int* Hb;
  const cplx* Ub;
  const cplx* weights;
  int* status;
};
bool ie_internal_factors(ie_handle h, IeFactorsView* v);

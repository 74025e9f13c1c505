// Harmonic Rayleigh-Ritz extraction "HSRR" (Sec. 2.1, extraction steps of Alg. SIsketch):
//   V = orth(U), W = orth(A V - sigma B V)   -- CGS2 with a rank guard
//   (W^* A V, W^* B V)                       -- Gram contractions over n
//   QZ: P_L^* (.) P_R = (H_A, H_B); lambda_i = (H_A)_ii / (H_B)_ii; x_i = V P_R V_R(:, i)
// plus the residuals e_i (Eq. rel-error) and rho_i, column permutation and seeded blocks.
#include "ie_internal.cuh"

namespace {
constexpr int OCH = 512;   // rows per chunk for the single-vector dot products

__device__ __forceinline__ cplx warp_sum_c(cplx v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), used counter-based: value = mix(seed + i*gamma).
__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double u01(uint64_t z) {   // (0, 1]
  return ((double)(z >> 11) + 1.0) * (1.0 / 9007199254740992.0);
}
// complex standard Gaussian entry (Box-Muller) for counter (seed, salt, col, row)
__device__ __forceinline__ cplx gauss_c(uint64_t seed, uint32_t salt, int64_t col, int64_t row) {
  const uint64_t base = splitmix64(seed ^ ((uint64_t)salt << 32) ^ 0x5DEECE66Dull);
  const uint64_t ctr = (uint64_t)col * 0x100000001B3ull + (uint64_t)row;
  const double a = u01(splitmix64(base + 2 * ctr));
  const double b = u01(splitmix64(base + 2 * ctr + 1));
  const double rad = sqrt(-2.0 * log(a));
  double sn, cs;
  sincospi(2.0 * b, &sn, &cs);
  return cmk(rad * cs, rad * sn);
}
}  // namespace

// ---------------- column-sequential CGS2 with rank guard ------------------------------------
// part[ch*LD + l] = sum_{r in chunk} conj(Q[r,l]) x[r] (l < j); part[ch*LD + j] = sum |x|^2.
// Skipped when gate != nullptr and *gate == 0.
__global__ void __launch_bounds__(256) odot_kernel(int64_t n, const cplx* Q, int64_t ldq, int j,
                                                   const cplx* x, cplx* part, int LD,
                                                   const int* gate) {
  if (gate && *gate == 0) return;
  const int ch = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t r0 = (int64_t)ch * OCH;
  cplx xr[OCH / 32];
#pragma unroll
  for (int u = 0; u < OCH / 32; ++u) {
    const int64_t r = r0 + lane + 32 * u;
    xr[u] = (r < n) ? x[r] : cmk(0, 0);
  }
  cplx* out = part + (int64_t)ch * LD;
  for (int l = warp; l < j; l += nw) {
    const cplx* q = Q + (int64_t)l * ldq;
    cplx acc = cmk(0, 0);
#pragma unroll
    for (int u = 0; u < OCH / 32; ++u) {
      const int64_t r = r0 + lane + 32 * u;
      if (r < n) acc = cfma_conj(q[r], xr[u], acc);
    }
    acc = warp_sum_c(acc);
    if (lane == 0) out[l] = acc;
  }
  if (warp == nw - 1) {
    double s2 = 0.0;
#pragma unroll
    for (int u = 0; u < OCH / 32; ++u) s2 += cabs2(xr[u]);
    s2 = warp_sum_d(s2);
    if (lane == 0) out[j] = cmk(s2, 0.0);
  }
}
__global__ void odot_reduce_kernel(int j, const cplx* part, int nchunk, int LD, cplx* h,
                                   const int* gate) {
  if (gate && *gate == 0) return;
  for (int l = threadIdx.x; l <= j; l += blockDim.x) {
    cplx t = cmk(0, 0);
    for (int ch = 0; ch < nchunk; ++ch) t = cadd(t, part[(int64_t)ch * LD + l]);
    h[l] = t;
  }
}
// x -= Q[:, :j] h
__global__ void oupdate_kernel(int64_t n, const cplx* Q, int64_t ldq, int j, cplx* x,
                               const cplx* h, const int* gate) {
  if (gate && *gate == 0) return;
  __shared__ cplx hs[1024];
  for (int l = threadIdx.x; l < j; l += blockDim.x) hs[l] = h[l];
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  cplx acc = cmk(0, 0);
  for (int l = 0; l < j; ++l) acc = cfma(Q[(int64_t)l * ldq + r], hs[l], acc);
  x[r] = csub(x[r], acc);
}
// Rank guard (decided identically by every thread): nrm0sq = ||x||^2 before projection,
// h_last[j].x = ||x||^2 after the two projections. If the column vanished (zero, or
// <= 1e-12 of its original norm) it is replaced by a seeded random vector and *flag = 1,
// which enables the two gated projection passes that follow.
__global__ void oguard_kernel(int64_t n, int j, const double* nrm0sq, const cplx* h_last, cplx* x,
                              uint64_t seed, uint32_t salt, int* flag) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double n0 = sqrt(*nrm0sq);
  const double n1 = sqrt(h_last[j].x);
  const bool rep = (n0 == 0.0) || (n1 <= 1e-12 * n0);
  if (r == 0) *flag = rep ? 1 : 0;
  if (rep && r < n) x[r] = gauss_c(seed, salt, j, r);
}
__global__ void onormalize_kernel(int64_t n, int j, const cplx* h_norm, cplx* x) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double nr = sqrt(h_norm[j].x);
  x[r] = (nr > 0.0) ? cscale(x[r], 1.0 / nr) : cmk(0, 0);
}
__global__ void copy_scalar_kernel(const cplx* src, double* dst) { *dst = src->x; }

void launch_orth_cgs2(int64_t n, int k, cplx* Q, int64_t ldq, uint64_t seed, uint32_t salt,
                      cplx* hbuf, double* scratch, int* flags, cudaStream_t s) {
  // hbuf: 3 vectors of length k+1 (h pass 1, h pass 2, final norm); scratch: nchunk*(k+1) cplx
  const int nchunk = (int)((n + OCH - 1) / OCH);
  const int LD = k + 1;
  cplx* part = (cplx*)scratch;
  cplx* h1 = hbuf;
  cplx* h2 = hbuf + LD;
  cplx* h3 = hbuf + 2 * LD;
  double* nrm0 = (double*)(hbuf + 3 * LD);
  const unsigned nb = (unsigned)((n + 255) / 256);
  for (int j = 0; j < k; ++j) {
    cplx* x = Q + (int64_t)j * ldq;
    // pass 1 (its norm slot = ||x||^2 before projection)
    odot_kernel<<<nchunk, 256, 0, s>>>(n, Q, ldq, j, x, part, LD, nullptr); ie_count_launch();
    odot_reduce_kernel<<<1, 256, 0, s>>>(j, part, nchunk, LD, h1, nullptr); ie_count_launch();
    copy_scalar_kernel<<<1, 1, 0, s>>>(h1 + j, nrm0); ie_count_launch();
    if (j > 0) oupdate_kernel<<<nb, 256, 0, s>>>(n, Q, ldq, j, x, h1, nullptr); ie_count_launch();
    // pass 2
    odot_kernel<<<nchunk, 256, 0, s>>>(n, Q, ldq, j, x, part, LD, nullptr); ie_count_launch();
    odot_reduce_kernel<<<1, 256, 0, s>>>(j, part, nchunk, LD, h2, nullptr); ie_count_launch();
    if (j > 0) oupdate_kernel<<<nb, 256, 0, s>>>(n, Q, ldq, j, x, h2, nullptr); ie_count_launch();
    // norm after the two passes
    odot_kernel<<<nchunk, 256, 0, s>>>(n, Q, ldq, 0, x, part, LD, nullptr); ie_count_launch();
    odot_reduce_kernel<<<1, 256, 0, s>>>(0, part, nchunk, LD, h3 + j, nullptr); ie_count_launch();
    // rank guard: replace by a seeded random vector, then project it twice (gated)
    oguard_kernel<<<nb, 256, 0, s>>>(n, j, nrm0, h3, x, seed, salt, flags + j); ie_count_launch();
    for (int pass = 0; pass < 2; ++pass) {
      odot_kernel<<<nchunk, 256, 0, s>>>(n, Q, ldq, j, x, part, LD, flags + j); ie_count_launch();
      odot_reduce_kernel<<<1, 256, 0, s>>>(j, part, nchunk, LD, h1, flags + j); ie_count_launch();
      if (j > 0) oupdate_kernel<<<nb, 256, 0, s>>>(n, Q, ldq, j, x, h1, flags + j); ie_count_launch();
    }
    odot_kernel<<<nchunk, 256, 0, s>>>(n, Q, ldq, 0, x, part, LD, flags + j); ie_count_launch();
    odot_reduce_kernel<<<1, 256, 0, s>>>(0, part, nchunk, LD, h3 + j, flags + j); ie_count_launch();
    onormalize_kernel<<<nb, 256, 0, s>>>(n, j, h3, x); ie_count_launch();
  }
}

// ---------------- Gram contraction C = W^H Y (k x k) -----------------------------------------
// Block = 32x32 output tile over a chunk of GCH rows, 256 threads with 2x2 outputs each;
// partials per chunk, then a deterministic reduction.
constexpr int GCH = 512;
__global__ void __launch_bounds__(256) gram_part_kernel(int64_t n, int k, const cplx* W,
                                                        int64_t ldw, const cplx* Y, int64_t ldy,
                                                        cplx* part) {
  const int ta = blockIdx.x * 32, tb = blockIdx.y * 32, ch = blockIdx.z;
  __shared__ cplx Ws[16][33], Ys[16][33];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  cplx acc[2][2] = {{cmk(0, 0), cmk(0, 0)}, {cmk(0, 0), cmk(0, 0)}};
  const int64_t rbeg = (int64_t)ch * GCH;
  const int64_t rend = (rbeg + GCH < n) ? (rbeg + GCH) : n;
  for (int64_t r0 = rbeg; r0 < rend; r0 += 16) {
    for (int e = threadIdx.x; e < 16 * 32; e += 256) {
      const int rr = e & 15, cc = e >> 4;
      const int64_t r = r0 + rr;
      Ws[rr][cc] = (r < rend && ta + cc < k) ? W[(int64_t)(ta + cc) * ldw + r] : cmk(0, 0);
      Ys[rr][cc] = (r < rend && tb + cc < k) ? Y[(int64_t)(tb + cc) * ldy + r] : cmk(0, 0);
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < 16; ++rr) {
      const cplx w0 = Ws[rr][tx], w1 = Ws[rr][tx + 16];
      const cplx y0 = Ys[rr][ty], y1 = Ys[rr][ty + 16];
      acc[0][0] = cfma_conj(w0, y0, acc[0][0]);
      acc[0][1] = cfma_conj(w0, y1, acc[0][1]);
      acc[1][0] = cfma_conj(w1, y0, acc[1][0]);
      acc[1][1] = cfma_conj(w1, y1, acc[1][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int a = ta + tx + 16 * u, b = tb + ty + 16 * v;
      if (a < k && b < k) part[((int64_t)ch * k + b) * k + a] = acc[u][v];
    }
}
__global__ void gram_reduce_kernel(int k, const cplx* part, int nchunk, cplx* C) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  cplx t = cmk(0, 0);
  for (int ch = 0; ch < nchunk; ++ch) t = cadd(t, part[(int64_t)ch * k * k + e]);
  C[e] = t;
}
void launch_gram(int64_t n, int k, const cplx* W, int64_t ldw, const cplx* Y, int64_t ldy,
                 cplx* C, cplx* scratch, cudaStream_t s) {
  const int nchunk = (int)((n + GCH - 1) / GCH);
  const int tiles = (k + 31) / 32;
  gram_part_kernel<<<dim3(tiles, tiles, nchunk), 256, 0, s>>>(n, k, W, ldw, Y, ldy, scratch); ie_count_launch();
  gram_reduce_kernel<<<(k * k + 255) / 256, 256, 0, s>>>(k, scratch, nchunk, C); ie_count_launch();
}

// ---------------- complex QZ (one CTA) --------------------------------------------------------
// Moler & Stewart's QZ for complex pencils: B to triangular (Givens QR), (A, B) to
// Hessenberg-triangular, single-shift QZ sweeps with deflation, zero-diagonal-of-B chasing
// (infinite eigenvalues), then right eigenvectors of the triangular pair by back substitution,
// transformed by Z (= P_R). Every rotation is computed redundantly by all threads from shared
// values, then applied in parallel; two barriers per rotation.
namespace {
__device__ __forceinline__ void qz_givens(cplx a, cplx b, double& c, cplx& s) {
  const double aa = cabsv(a), bb = cabsv(b);
  if (bb == 0.0) { c = 1.0; s = cmk(0, 0); }
  else if (aa == 0.0) { c = 0.0; s = cscale(cconj(b), 1.0 / bb); }
  else {
    const double nu = hypot(aa, bb);
    c = aa / nu;
    s = cmul(cscale(a, 1.0 / aa), cscale(cconj(b), 1.0 / nu));
  }
}
// rows r1, r2, columns c0..k-1: [x; y] <- [c x + s y; -conj(s) x + c y]
__device__ __forceinline__ void qz_row(cplx* M, int k, int r1, int r2, int c0, double c, cplx s) {
  for (int j = c0 + (int)threadIdx.x; j < k; j += blockDim.x) {
    const cplx x = M[r1 + j * k], y = M[r2 + j * k];
    M[r1 + j * k] = cadd(cscale(x, c), cmul(s, y));
    M[r2 + j * k] = cadd(cmul(cmk(-s.x, s.y), x), cscale(y, c));
  }
}
// columns c1, c2, rows 0..r1: [x, y] <- [c x - conj(s) y, s x + c y]
__device__ __forceinline__ void qz_col(cplx* M, int k, int c1, int c2, int r1, double c, cplx s) {
  for (int i = (int)threadIdx.x; i <= r1; i += blockDim.x) {
    const cplx x = M[i + c1 * k], y = M[i + c2 * k];
    M[i + c1 * k] = csub(cscale(x, c), cmul(cconj(s), y));
    M[i + c2 * k] = cadd(cmul(s, x), cscale(y, c));
  }
}
__device__ cplx csqrt_(cplx z) {
  const double r = cabsv(z);
  if (r == 0.0) return cmk(0, 0);
  const double w = sqrt(0.5 * (r + fabs(z.x)));
  if (z.x >= 0.0) return cmk(w, z.y / (2.0 * w));
  return cmk(fabs(z.y) / (2.0 * w), (z.y >= 0.0) ? w : -w);
}
}  // namespace

__global__ void __launch_bounds__(256) qz_kernel(int k, cplx* gA, cplx* gB, cplx* gZ, cplx* alpha,
                                                 cplx* beta, cplx* Mout, cplx* VR, int* status,
                                                 int use_smem) {
  extern __shared__ double2 qz_sm[];
  cplx *A, *B, *Z;
  const int tid = threadIdx.x, T = blockDim.x;
  if (use_smem) {
    A = qz_sm; B = A + k * k; Z = B + k * k;
    for (int e = tid; e < k * k; e += T) { A[e] = gA[e]; B[e] = gB[e]; }
  } else {
    A = gA; B = gB; Z = gZ;
  }
  for (int e = tid; e < k * k; e += T) Z[e] = cmk((e % k) == (e / k) ? 1.0 : 0.0, 0.0);
  __shared__ double red[32];
  double sa = 0.0, sb = 0.0;
  for (int e = tid; e < k * k; e += T) { sa += cabs2(A[e]); sb += cabs2(B[e]); }
  sa = warp_sum_d(sa); sb = warp_sum_d(sb);
  __shared__ double s_an, s_bn;
  if ((tid & 31) == 0) red[tid >> 5] = sa;
  __syncthreads();
  if (tid == 0) { double t = 0; for (int w = 0; w < T / 32; ++w) t += red[w]; s_an = sqrt(t); }
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = sb;
  __syncthreads();
  if (tid == 0) { double t = 0; for (int w = 0; w < T / 32; ++w) t += red[w]; s_bn = sqrt(t); }
  __syncthreads();
  const double anorm = s_an, bnorm = s_bn;
  const double ulp = 2.220446049250313e-16;
#define QA(i, j) A[(i) + (j) * k]
#define QB(i, j) B[(i) + (j) * k]
  double c; cplx s;
  // 1. B = Q R by Givens; A <- Q^H A
  for (int j = 0; j < k - 1; ++j)
    for (int i = k - 1; i > j; --i) {
      const cplx bb = QB(i, j);
      if (bb.x == 0.0 && bb.y == 0.0) continue;
      qz_givens(QB(i - 1, j), bb, c, s);
      __syncthreads();
      qz_row(B, k, i - 1, i, j, c, s);
      qz_row(A, k, i - 1, i, 0, c, s);
      __syncthreads();
      if (tid == 0) QB(i, j) = cmk(0, 0);
      __syncthreads();
    }
  // 2. Hessenberg-triangular reduction
  for (int j = 0; j + 2 < k; ++j)
    for (int i = k - 1; i >= j + 2; --i) {
      const cplx aa = QA(i, j);
      if (aa.x != 0.0 || aa.y != 0.0) {
        qz_givens(QA(i - 1, j), aa, c, s);
        __syncthreads();
        qz_row(A, k, i - 1, i, j, c, s);
        qz_row(B, k, i - 1, i, i - 1, c, s);
        __syncthreads();
        if (tid == 0) QA(i, j) = cmk(0, 0);
        __syncthreads();
      }
      const cplx bb = QB(i, i - 1);
      if (bb.x != 0.0 || bb.y != 0.0) {
        qz_givens(QB(i, i), bb, c, s);
        __syncthreads();
        qz_col(A, k, i - 1, i, k - 1, c, s);
        qz_col(B, k, i - 1, i, i, c, s);
        qz_col(Z, k, i - 1, i, k - 1, c, s);
        __syncthreads();
        if (tid == 0) QB(i, i - 1) = cmk(0, 0);
        __syncthreads();
      }
    }
  // 3. QZ iterations
  int ihi = k - 1, iter = 0, total = 0;
  bool fail = false;
  while (ihi > 0) {
    int ilo = 0;
    for (int i = ihi; i >= 1; --i) {
      const double sub = cabs1(QA(i, i - 1));
      if (sub <= ulp * (cabs1(QA(i, i)) + cabs1(QA(i - 1, i - 1))) || sub <= ulp * anorm * 1e-2) {
        ilo = i;
        break;
      }
    }
    __syncthreads();
    if (ilo > 0 && tid == 0) QA(ilo, ilo - 1) = cmk(0, 0);
    __syncthreads();
    if (ilo == ihi) { --ihi; iter = 0; continue; }
    int jz = -1;
    for (int jj = ilo; jj <= ihi; ++jj)
      if (cabsv(QB(jj, jj)) <= ulp * bnorm) { jz = jj; break; }
    __syncthreads();
    if (jz >= 0) {
      if (tid == 0) QB(jz, jz) = cmk(0, 0);
      __syncthreads();
      for (int i = jz; i < ihi; ++i) {
        qz_givens(QB(i, i + 1), QB(i + 1, i + 1), c, s);
        __syncthreads();
        qz_row(B, k, i, i + 1, i + 1, c, s);
        qz_row(A, k, i, i + 1, (i > ilo) ? i - 1 : ilo, c, s);
        __syncthreads();
        if (tid == 0) QB(i + 1, i + 1) = cmk(0, 0);
        __syncthreads();
        if (i > ilo) {
          qz_givens(QA(i + 1, i), QA(i + 1, i - 1), c, s);
          __syncthreads();
          qz_col(A, k, i - 1, i, i + 1, c, s);
          qz_col(B, k, i - 1, i, i, c, s);
          qz_col(Z, k, i - 1, i, k - 1, c, s);
          __syncthreads();
          if (tid == 0) QA(i + 1, i - 1) = cmk(0, 0);
          __syncthreads();
        }
      }
      qz_givens(QA(ihi, ihi), QA(ihi, ihi - 1), c, s);
      __syncthreads();
      qz_col(A, k, ihi - 1, ihi, ihi, c, s);
      qz_col(B, k, ihi - 1, ihi, ihi, c, s);
      qz_col(Z, k, ihi - 1, ihi, k - 1, c, s);
      __syncthreads();
      if (tid == 0) QA(ihi, ihi - 1) = cmk(0, 0);
      __syncthreads();
      --ihi;
      iter = 0;
      continue;
    }
    ++iter;
    if (++total > 40 * k) { fail = true; break; }
    // shift: eigenvalue of the trailing 2x2 pencil closest to a22/b22
    const cplx a11 = QA(ihi - 1, ihi - 1), a12 = QA(ihi - 1, ihi), a21 = QA(ihi, ihi - 1),
               a22 = QA(ihi, ihi);
    const cplx b11 = QB(ihi - 1, ihi - 1), b12 = QB(ihi - 1, ihi), b22 = QB(ihi, ihi);
    const cplx ref = cdiv(a22, b22);
    cplx mu;
    if (iter % 10 == 0) {
      const double sc = cabsv(a21) / fmax(cabsv(b11), 1e-300);
      mu = cadd(ref, cscale(cmk(0.75, 0.5), sc));
    } else {
      const cplx qa = cmul(b11, b22);
      const cplx qb = csub(cmul(a21, b12), cadd(cmul(a11, b22), cmul(a22, b11)));
      const cplx qc = csub(cmul(a11, a22), cmul(a12, a21));
      if (cabsv(qa) <= ulp * (cabsv(qb) + cabsv(qc))) {
        mu = ref;
      } else {
        const cplx disc = csqrt_(csub(cmul(qb, qb), cscale(cmul(qa, qc), 4.0)));
        cplx qq = cadd(qb, disc);
        const cplx qm = csub(qb, disc);
        if (cabsv(qm) > cabsv(qq)) qq = qm;
        qq = cscale(qq, -0.5);
        const cplx r1 = cdiv(qq, qa);
        const cplx r2 = (cabsv(qq) > 0.0) ? cdiv(qc, qq) : r1;
        mu = (cabsv(csub(r1, ref)) <= cabsv(csub(r2, ref))) ? r1 : r2;
      }
    }
    const cplx x = csub(cdiv(QA(ilo, ilo), QB(ilo, ilo)), mu);
    const cplx y = cdiv(QA(ilo + 1, ilo), QB(ilo, ilo));
    qz_givens(x, y, c, s);
    __syncthreads();
    qz_row(A, k, ilo, ilo + 1, ilo, c, s);
    qz_row(B, k, ilo, ilo + 1, ilo, c, s);
    __syncthreads();
    for (int i = ilo; i < ihi; ++i) {
      qz_givens(QB(i + 1, i + 1), QB(i + 1, i), c, s);
      __syncthreads();
      qz_col(A, k, i, i + 1, min(i + 2, ihi), c, s);
      qz_col(B, k, i, i + 1, i + 1, c, s);
      qz_col(Z, k, i, i + 1, k - 1, c, s);
      __syncthreads();
      if (tid == 0) QB(i + 1, i) = cmk(0, 0);
      __syncthreads();
      if (i < ihi - 1) {
        qz_givens(QA(i + 1, i), QA(i + 2, i), c, s);
        __syncthreads();
        qz_row(A, k, i + 1, i + 2, i, c, s);
        qz_row(B, k, i + 1, i + 2, i + 1, c, s);
        __syncthreads();
        if (tid == 0) QA(i + 2, i) = cmk(0, 0);
        __syncthreads();
      }
    }
  }
  if (fail && tid == 0) atomicExch(status + 3, 1);
  __syncthreads();
  // 4. eigenvalues, 5. right eigenvectors of the triangular pair (thread per eigenvalue)
  double amax = 0.0, bmax = 0.0;
  for (int e = 0; e < k * k; ++e) { amax = fmax(amax, cabsv(A[e])); bmax = fmax(bmax, cabsv(B[e])); }
  for (int i = tid; i < k; i += T) {
    const cplx al = QA(i, i), be = QB(i, i);
    alpha[i] = al;
    beta[i] = be;
    const double small = ulp * (cabsv(be) * amax + cabsv(al) * bmax);
    cplx* v = VR + (int64_t)i * k;
    for (int jj = i + 1; jj < k; ++jj) v[jj] = cmk(0, 0);
    v[i] = cmk(1.0, 0.0);
    for (int jj = i - 1; jj >= 0; --jj) {
      cplx acc = cmk(0, 0);
      for (int l = jj + 1; l <= i; ++l) {
        const cplx m = csub(cmul(be, QA(jj, l)), cmul(al, QB(jj, l)));
        acc = cfma(m, v[l], acc);
      }
      cplx d = csub(cmul(be, QA(jj, jj)), cmul(al, QB(jj, jj)));
      if (cabsv(d) <= small) d = cmk(small > 0.0 ? small : ulp, 0.0);
      v[jj] = cdiv(cscale(acc, -1.0), d);
    }
  }
  __syncthreads();
  // M = Z VR
  for (int e = tid; e < k * k; e += T) {
    const int r = e % k, cc = e / k;
    cplx acc = cmk(0, 0);
    for (int l = 0; l <= cc; ++l) acc = cfma(Z[r + l * k], VR[(int64_t)cc * k + l], acc);
    Mout[e] = acc;
  }
#undef QA
#undef QB
}

cudaError_t launch_qz(int k, cplx* Ah, cplx* Bh, cplx* Z, cplx* alpha, cplx* beta, cplx* M,
                      int* status, cudaStream_t s) {
  // VR scratch placed after Z (caller allocates 2*k*k for Z)
  cplx* VR = Z + (int64_t)k * k;
  const size_t smem = (size_t)3 * k * k * sizeof(cplx);
  const int use_smem = smem <= 200 * 1024;
  if (use_smem) {
    cudaError_t e = ie_smem_optin((const void*)qz_kernel);
    if (e != cudaSuccess) return e;
  }
  qz_kernel<<<1, 256, use_smem ? smem : 0, s>>>(k, Ah, Bh, Z, alpha, beta, M, VR, status,
                                                use_smem); ie_count_launch();
  return cudaGetLastError();
}

// ---------------- small GEMM, normalisation, residuals, permutation, random ------------------
__global__ void gemm_small_kernel(int64_t n, int k, const cplx* X, int64_t ldx, const cplx* M,
                                  cplx* Y, int64_t ldy) {
  const int c = blockIdx.y;
  __shared__ cplx ms[256];
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  cplx acc = cmk(0, 0);
  for (int l0 = 0; l0 < k; l0 += 256) {
    __syncthreads();
    for (int l = threadIdx.x; l < 256 && l0 + l < k; l += blockDim.x)
      ms[l] = M[(int64_t)c * k + l0 + l];
    __syncthreads();
    if (r < n) {
      const int lend = min(256, k - l0);
      for (int l = 0; l < lend; ++l) acc = cfma(X[(int64_t)(l0 + l) * ldx + r], ms[l], acc);
    }
  }
  if (r < n) Y[(int64_t)c * ldy + r] = acc;
}
void launch_gemm_small(int64_t n, int k, const cplx* X, int64_t ldx, const cplx* M, cplx* Y,
                       int64_t ldy, cudaStream_t s) {
  gemm_small_kernel<<<dim3((unsigned)((n + 255) / 256), k), 256, 0, s>>>(n, k, X, ldx, M, Y, ldy); ie_count_launch();
}

__global__ void scale_cols_kernel(int64_t n, cplx* X, int64_t ldx, const double* nrm) {
  const int c = blockIdx.y;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const double v = nrm[c];
  if (v > 0.0) X[(int64_t)c * ldx + r] = cscale(X[(int64_t)c * ldx + r], 1.0 / v);
}
void launch_normalize_cols(int64_t n, int k, cplx* X, int64_t ldx, double* scratch,
                           cudaStream_t s) {
  double* nrm = scratch;
  launch_colnorm2(n, k, X, ldx, nrm, scratch + k, s);
  scale_cols_kernel<<<dim3((unsigned)((n + 255) / 256), k), 256, 0, s>>>(n, X, ldx, nrm); ie_count_launch();
}

__global__ void resid_part_kernel(DiaDev P, const cplx* X, int64_t ldx, const cplx* lam,
                                  double* part, int nblk) {
  const int c = blockIdx.y;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double r2 = 0.0, b2 = 0.0, x2 = 0.0;
  const cplx* x = X + (int64_t)c * ldx;
  const cplx l = lam[c];
  const bool finite = isfinite(l.x) && isfinite(l.y);
  if (i < P.n) {
    cplx ax = cmk(0, 0), bx = cmk(0, 0);
    for (int d = 0; d < P.ndiag; ++d) {
      const int64_t j = i + P.off[d];
      if (j < 0 || j >= P.n) continue;
      const cplx xv = x[j];
      ax = cfma(P.A[(int64_t)d * P.n + i], xv, ax);
      bx = cfma(P.B[(int64_t)d * P.n + i], xv, bx);
    }
    const cplx r = finite ? cfms(l, bx, ax) : cmk(0, 0);
    r2 = cabs2(r);
    b2 = cabs2(bx);
    x2 = cabs2(x[i]);
  }
  r2 = warp_sum_d(r2); b2 = warp_sum_d(b2); x2 = warp_sum_d(x2);
  __shared__ double sm[3][32];
  if ((threadIdx.x & 31) == 0) { sm[0][threadIdx.x >> 5] = r2; sm[1][threadIdx.x >> 5] = b2; sm[2][threadIdx.x >> 5] = x2; }
  __syncthreads();
  if (threadIdx.x < 3) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[threadIdx.x][w];
    part[((int64_t)c * nblk + blockIdx.x) * 3 + threadIdx.x] = t;
  }
}
__global__ void resid_reduce_kernel(int k, const double* part, int nblk, double* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * k) return;
  const int c = t / 3, w = t % 3;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += part[((int64_t)c * nblk + b) * 3 + w];
  out[t] = s;
}
void launch_residual_norms(const DiaDev& P, int k, const cplx* X, int64_t ldx, const cplx* lam,
                           double* d_out, double* scratch, cudaStream_t s) {
  const int nblk = (int)((P.n + 255) / 256);
  resid_part_kernel<<<dim3(nblk, k), 256, 0, s>>>(P, X, ldx, lam, scratch, nblk); ie_count_launch();
  resid_reduce_kernel<<<(3 * k + 127) / 128, 128, 0, s>>>(k, scratch, nblk, d_out); ie_count_launch();
}

__global__ void permute_cols_kernel(int64_t n, const cplx* X, int64_t ldx, const int* perm,
                                    cplx* Y, int64_t ldy) {
  const int c = blockIdx.y;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) Y[(int64_t)c * ldy + r] = X[(int64_t)perm[c] * ldx + r];
}
void launch_permute_cols(int64_t n, int k, const cplx* X, int64_t ldx, const int* perm, cplx* Y,
                         int64_t ldy, cudaStream_t s) {
  permute_cols_kernel<<<dim3((unsigned)((n + 255) / 256), k), 256, 0, s>>>(n, X, ldx, perm, Y,
                                                                           ldy); ie_count_launch();
}

__global__ void random_block_kernel(int64_t n, cplx* X, int64_t ldx, uint64_t seed,
                                    uint32_t salt) {
  const int c = blockIdx.y;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) X[(int64_t)c * ldx + r] = gauss_c(seed, salt, c, r);
}
void launch_random_block(int64_t n, int k, cplx* X, int64_t ldx, uint64_t seed, uint32_t salt,
                         cudaStream_t s) {
  random_block_kernel<<<dim3((unsigned)((n + 255) / 256), k), 256, 0, s>>>(n, X, ldx, seed, salt); ie_count_launch();
}

__global__ void copy_cols_kernel(int64_t n, const cplx* X, int64_t ldx, cplx* Y, int64_t ldy) {
  const int c = blockIdx.y;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) Y[(int64_t)c * ldy + r] = X[(int64_t)c * ldx + r];
}
void launch_copy_cols(int64_t n, int k, const cplx* X, int64_t ldx, cplx* Y, int64_t ldy,
                      cudaStream_t s) {
  if (k <= 0) return;
  copy_cols_kernel<<<dim3((unsigned)((n + 255) / 256), k), 256, 0, s>>>(n, X, ldx, Y, ldy); ie_count_launch();
}

// Outer rational function by multi-shift GMRES (Sec. 3.2, Eq. linearsolve1abs; filter step
// of Alg. 1): one Arnoldi basis of G per column, orthogonalised by CGS2 (classical Gram-Schmidt,
// twice), shared by all outer shifts s_j, since (G - sI) V_J = V_{J+1} (Hbar_J - s Ibar_J).
// Per (column, shift) the QR factorisation of Hbar - s Ibar is updated by Givens rotations;
// the last rotated right-hand-side entry is the GMRES residual.
#include "ie_internal.cuh"

namespace {
constexpr int CH = 512;   // rows per chunk of the batched dot products (16 per lane)

__device__ __forceinline__ cplx warp_sum(cplx v) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
}  // namespace

// ---------------- column norms ----------------------------------------------------------------
__global__ void colnorm2_part_kernel(int64_t n, const cplx* X, int64_t ldx, double* part,
                                     int nchunk) {
  const int c = blockIdx.y, ch = blockIdx.x;
  const cplx* x = X + (int64_t)c * ldx;
  double s = 0.0;
  for (int64_t r = (int64_t)ch * blockDim.x + threadIdx.x; r < n; r += (int64_t)nchunk * blockDim.x)
    s += cabs2(x[r]);
  s = warp_sum(s);
  __shared__ double sm[32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
    part[(int64_t)c * nchunk + ch] = t;
  }
}
__global__ void sum_parts_sqrt_kernel(int k, const double* part, int nchunk, double* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  double t = 0.0;
  for (int i = 0; i < nchunk; ++i) t += part[(int64_t)c * nchunk + i];
  out[c] = sqrt(t);
}
static int colnorm_chunks(int64_t n) {
  int64_t c = (n + 255) / 256;
  return (int)(c > 64 ? 64 : (c < 1 ? 1 : c));
}
void launch_colnorm2(int64_t n, int k, const cplx* X, int64_t ldx, double* d_out,
                     double* d_scratch, cudaStream_t s) {
  if (k <= 0) return;
  const int nchunk = colnorm_chunks(n);
  colnorm2_part_kernel<<<dim3(nchunk, k), 256, 0, s>>>(n, X, ldx, d_scratch, nchunk); ie_count_launch();
  sum_parts_sqrt_kernel<<<(k + 127) / 128, 128, 0, s>>>(k, d_scratch, nchunk, d_out); ie_count_launch();
}

// ---------------- Krylov start: beta_c = ||ytilde_c||, v_0 = ytilde_c / beta_c -----------------
__global__ void krylov_start_kernel(KrylovDev K, const cplx* Yt, int64_t ldy) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  const double b = K.beta[c];
  if (r < K.n) {
    const cplx y = Yt[(int64_t)c * ldy + r];
    K.V[(int64_t)c * (K.m_max + 1) * K.n + r] = (b > 0.0) ? cscale(y, 1.0 / b) : cmk(0, 0);
  }
  if (r == 0) {
    K.jc[c] = 0;
    K.brk[c] = (b > 0.0) ? 0 : 1;
  }
}
void launch_krylov_start(const KrylovDev& K, int k, const cplx* Yt, int64_t ldy, double* scratch,
                         cudaStream_t s) {
  launch_colnorm2(K.n, k, Yt, ldy, K.beta, scratch, s);
  krylov_start_kernel<<<dim3((unsigned)((K.n + 255) / 256), k), 256, 0, s>>>(K, Yt, ldy); ie_count_launch();
}

__global__ void active_offsets_kernel(KrylovDev K, const int* act, int kact, int64_t* off) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kact) return;
  const int c = act[i];
  off[i] = ((int64_t)c * (K.m_max + 1) + K.jc[c]) * K.n;
}
void launch_active_offsets(const KrylovDev& K, const int* act, int kact, int64_t* d_off,
                           cudaStream_t s) {
  if (kact <= 0) return;
  active_offsets_kernel<<<(kact + 127) / 128, 128, 0, s>>>(K, act, kact, d_off); ie_count_launch();
}

// ---------------- CGS2 Arnoldi step ---------------------------------------------------------
// part[(i*nchunk + ch)*LD + l] = sum_{r in chunk} conj(V_c[r,l]) w_i[r], l = 0..j;
// with want_norm, part[..+ j+1] = sum |w_i[r]|^2. One warp per basis vector l (strided by warps),
// lanes over the chunk's rows (coalesced); the chunk of w sits in registers.
__global__ void __launch_bounds__(256) mdot_kernel(KrylovDev K, const int* act, const cplx* W,
                                                   int64_t ldw, double* part, int nchunk, int LD,
                                                   int want_norm) {
  const int i = blockIdx.y, ch = blockIdx.x;
  const int c = act[i];
  const int j = K.jc[c];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t r0 = (int64_t)ch * CH;
  const cplx* w = W + (int64_t)i * ldw;
  cplx wr[CH / 32];
#pragma unroll
  for (int u = 0; u < CH / 32; ++u) {
    const int64_t r = r0 + lane + 32 * u;
    wr[u] = (r < K.n) ? w[r] : cmk(0, 0);
  }
  const cplx* Vc = K.V + (int64_t)c * (K.m_max + 1) * K.n;
  cplx* out = (cplx*)(part) + ((int64_t)i * nchunk + ch) * LD;
  for (int l = warp; l <= j; l += nw) {
    const cplx* v = Vc + (int64_t)l * K.n;
    cplx acc = cmk(0, 0);
#pragma unroll
    for (int u = 0; u < CH / 32; ++u) {
      const int64_t r = r0 + lane + 32 * u;
      if (r < K.n) acc = cfma_conj(v[r], wr[u], acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) out[l] = acc;
  }
  if (want_norm && warp == nw - 1) {
    double s2 = 0.0;
#pragma unroll
    for (int u = 0; u < CH / 32; ++u) s2 += cabs2(wr[u]);
    s2 = warp_sum(s2);
    if (lane == 0) out[j + 1] = cmk(s2, 0.0);
  }
}

// h[i*LD + l] = sum_ch part[(i*nchunk+ch)*LD + l] for l <= j (+1 with the norm slot)
__global__ void mdot_reduce_kernel(KrylovDev K, const int* act, const double* part, int nchunk,
                                   int LD, cplx* h, int with_norm) {
  const int i = blockIdx.x;
  const int c = act[i];
  const int j = K.jc[c];
  const int lmax = j + (with_norm ? 1 : 0);
  const cplx* p = (const cplx*)part + (int64_t)i * nchunk * LD;
  for (int l = threadIdx.x; l <= lmax; l += blockDim.x) {
    cplx t = cmk(0, 0);
    for (int ch = 0; ch < nchunk; ++ch) t = cadd(t, p[(int64_t)ch * LD + l]);
    h[(int64_t)i * LD + l] = t;
  }
}

// w_i[r] -= sum_{l<=j} V_c[r,l] h[l]; optionally part2[i*nblk + blk] = sum |w_new|^2
__global__ void __launch_bounds__(256) mupdate_kernel(KrylovDev K, const int* act, cplx* W,
                                                      int64_t ldw, const cplx* h, int LD,
                                                      double* part2, int nblk) {
  const int i = blockIdx.y;
  const int c = act[i];
  const int j = K.jc[c];
  __shared__ cplx hs[1024];
  for (int l = threadIdx.x; l <= j; l += blockDim.x) hs[l] = h[(int64_t)i * LD + l];
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s2 = 0.0;
  if (r < K.n) {
    const cplx* Vc = K.V + (int64_t)c * (K.m_max + 1) * K.n;
    cplx acc = cmk(0, 0);
    for (int l = 0; l <= j; ++l) acc = cfma(Vc[(int64_t)l * K.n + r], hs[l], acc);
    cplx* w = W + (int64_t)i * ldw;
    const cplx nw = csub(w[r], acc);
    w[r] = nw;
    s2 = cabs2(nw);
  }
  if (part2) {
    s2 = warp_sum(s2);
    __shared__ double sm[32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s2;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sm[w];
      part2[(int64_t)i * nblk + blockIdx.x] = t;
    }
  }
}

// H_c[0..j, j] = h1 + h2; H_c[j+1, j] = ||w||; lucky breakdown if ||w|| <= 1e-14 ||G v_j||.
// scale[i] = 1/||w|| (0 on breakdown); jc[c] = j + 1.
__global__ void arnoldi_finish_kernel(KrylovDev K, const int* act, int kact, const cplx* h1,
                                      const cplx* h2, int LD, const double* part2, int nblk,
                                      double* scale) {
  const int i = blockIdx.x;
  if (i >= kact) return;
  const int c = act[i];
  const int j = K.jc[c];
  cplx* Hc = K.H + (int64_t)c * (K.m_max + 1) * K.m_max + (int64_t)j * (K.m_max + 1);
  for (int l = threadIdx.x; l <= j; l += blockDim.x)
    Hc[l] = cadd(h1[(int64_t)i * LD + l], h2[(int64_t)i * LD + l]);
  __shared__ double sm[32];
  double t = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) t += part2[(int64_t)i * nblk + b];
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s2 += sm[w];
    const double hn = sqrt(s2);
    const double wn0 = sqrt(h1[(int64_t)i * LD + j + 1].x);
    if (hn <= 1e-14 * wn0 || hn == 0.0) {
      Hc[j + 1] = cmk(0, 0);
      K.brk[c] = 1;
      scale[i] = 0.0;
    } else {
      Hc[j + 1] = cmk(hn, 0.0);
      scale[i] = 1.0 / hn;
    }
    K.jc[c] = j + 1;
  }
}

// V_c[:, jc[c]] = w_i * scale[i]
__global__ void arnoldi_normalize_kernel(KrylovDev K, const int* act, const cplx* W, int64_t ldw,
                                         const double* scale) {
  const int i = blockIdx.y;
  const int c = act[i];
  const int j1 = K.jc[c];
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= K.n || j1 > K.m_max) return;
  K.V[((int64_t)c * (K.m_max + 1) + j1) * K.n + r] = cscale(W[(int64_t)i * ldw + r], scale[i]);
}

void launch_arnoldi_cgs2(const KrylovDev& K, const int* act, int kact, cplx* W, int64_t ldw,
                         cplx* hbuf, double* scratch, cudaStream_t s) {
  if (kact <= 0) return;
  const int nchunk = (int)((K.n + CH - 1) / CH);
  const int LD = K.m_max + 2;
  const int nblk = (int)((K.n + 255) / 256);
  cplx* h1 = hbuf;
  cplx* h2 = hbuf + (int64_t)kact * LD;
  double* scale = (double*)(hbuf + 2 * (int64_t)kact * LD);
  double* part = scratch;                                   // kact*nchunk*LD complex
  double* part2 = scratch + 2 * (int64_t)kact * nchunk * LD; // kact*nblk doubles
  const dim3 gdot(nchunk, kact), gupd(nblk, kact);
  // pass 1: h1 = V^H w (+ ||w||^2), w -= V h1
  mdot_kernel<<<gdot, 256, 0, s>>>(K, act, W, ldw, part, nchunk, LD, 1); ie_count_launch();
  mdot_reduce_kernel<<<kact, 128, 0, s>>>(K, act, part, nchunk, LD, h1, 1); ie_count_launch();
  mupdate_kernel<<<gupd, 256, 0, s>>>(K, act, W, ldw, h1, LD, nullptr, nblk); ie_count_launch();
  // pass 2: h2 = V^H w, w -= V h2, ||w||^2
  mdot_kernel<<<gdot, 256, 0, s>>>(K, act, W, ldw, part, nchunk, LD, 0); ie_count_launch();
  mdot_reduce_kernel<<<kact, 128, 0, s>>>(K, act, part, nchunk, LD, h2, 0); ie_count_launch();
  mupdate_kernel<<<gupd, 256, 0, s>>>(K, act, W, ldw, h2, LD, part2, nblk); ie_count_launch();
  arnoldi_finish_kernel<<<kact, 256, 0, s>>>(K, act, kact, h1, h2, LD, part2, nblk, scale); ie_count_launch();
  arnoldi_normalize_kernel<<<gupd, 256, 0, s>>>(K, act, W, ldw, scale); ie_count_launch();
}

// ---------------- multi-shift Givens ---------------------------------------------------------
// Rotation G = [c s; -conj(s) c] (c real) with G [a; b] = [r; 0].
__device__ __forceinline__ void givens(cplx a, cplx b, double& c, cplx& s, cplx& r) {
  const double aa = cabsv(a), bb = cabsv(b);
  if (bb == 0.0) {
    c = 1.0; s = cmk(0, 0); r = a;
  } else if (aa == 0.0) {
    c = 0.0; s = cscale(cconj(b), 1.0 / bb); r = cmk(bb, 0.0);
  } else {
    const double nu = hypot(aa, bb);
    const cplx ph = cscale(a, 1.0 / aa);
    c = aa / nu;
    s = cmul(ph, cscale(cconj(b), 1.0 / nu));
    r = cscale(ph, nu);
  }
}

// One thread per (active column i, shift l). Processes H columns [from, J) of column c where
// J = jc[c]; from = 0 restarts the factorisation (g = beta e_1), else from = J - 1.
__global__ void givens_kernel(KrylovDev K, const int* act, int kact, const cplx* shifts,
                              int nshift, double* rc, cplx* rs, cplx* g, int from_zero,
                              unsigned long long* res_bits) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= kact * nshift) return;
  const int i = t / nshift, l = t % nshift;
  const int c = act[i];
  const int J = K.jc[c];
  const cplx sh = shifts[l];
  const int64_t st = (int64_t)c * nshift + l;
  double* cc = rc + st * K.m_max;
  cplx* ss = rs + st * K.m_max;
  cplx* gg = g + st * (K.m_max + 1);
  const double beta = K.beta[c];
  const cplx* Hc = K.H + (int64_t)c * (K.m_max + 1) * K.m_max;
  int from = from_zero ? 0 : J - 1;
  if (from < 0) from = 0;
  if (from == 0) {
    gg[0] = cmk(beta, 0.0);
  }
  double res = (beta > 0.0) ? 1.0 : 0.0;
  for (int jj = from; jj < J; ++jj) {
    const cplx* hcol = Hc + (int64_t)jj * (K.m_max + 1);
    cplx carry = hcol[0];
    if (jj == 0) carry = csub(carry, sh);
    for (int q = 0; q < jj; ++q) {
      cplx b = hcol[q + 1];
      if (q + 1 == jj) b = csub(b, sh);
      const double cq = cc[q];
      const cplx sq = ss[q];
      // new_a = c a + s b (R entry, not kept); carry = -conj(s) a + c b
      carry = cadd(cmul(cmk(-sq.x, sq.y), carry), cscale(b, cq));
    }
    double cn;
    cplx sn, rr;
    givens(carry, hcol[jj + 1], cn, sn, rr);
    cc[jj] = cn;
    ss[jj] = sn;
    const cplx gj = gg[jj];
    gg[jj] = cscale(gj, cn);
    const cplx gn = cmul(cmk(-sn.x, sn.y), gj);
    gg[jj + 1] = gn;
    res = (beta > 0.0) ? cabsv(gn) / beta : 0.0;
  }
  atomicMax(res_bits + i, (unsigned long long)__double_as_longlong(res));
}

void launch_givens(const KrylovDev& K, const int* act, int kact, const cplx* d_shifts,
                   int nshift, cplx* rot_c, cplx* rot_s, cplx* gvec, int from_zero,
                   double* d_res, cudaStream_t s) {
  if (kact <= 0 || nshift <= 0) return;
  cudaMemsetAsync(d_res, 0, sizeof(double) * kact, s);
  const int tot = kact * nshift;
  givens_kernel<<<(tot + 127) / 128, 128, 0, s>>>(K, act, kact, d_shifts, nshift, (double*)rot_c,
                                                  rot_s, gvec, from_zero,
                                                  (unsigned long long*)d_res); ie_count_launch();
}

// ---------------- combine: U_c = V_c z_c, z_c = -sum_l wt_l y_l (+ odd beta e_1) -------------
// y_l = argmin || beta e_1 - (Hbar - s_l Ibar) y || by Givens QR and back substitution.
__global__ void ls_solve_kernel(KrylovDev K, int k, const cplx* shifts, int nshift, double* rc,
                                cplx* rs, cplx* R, cplx* y) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= k * nshift) return;
  const int c = t / nshift, l = t % nshift;
  const int J = K.jc[c];
  const int M = K.m_max;
  const cplx sh = shifts[l];
  const int64_t st = (int64_t)c * nshift + l;
  double* cc = rc + st * M;
  cplx* ss = rs + st * M;
  cplx* Rm = R + st * (int64_t)M * M;    // column-major, ld M
  cplx* yy = y + st * (M + 1);           // g, then y
  const double beta = K.beta[c];
  const cplx* Hc = K.H + (int64_t)c * (M + 1) * M;
  yy[0] = cmk(beta, 0.0);
  for (int jj = 0; jj < J; ++jj) {
    const cplx* hcol = Hc + (int64_t)jj * (M + 1);
    cplx carry = hcol[0];
    if (jj == 0) carry = csub(carry, sh);
    for (int q = 0; q < jj; ++q) {
      cplx b = hcol[q + 1];
      if (q + 1 == jj) b = csub(b, sh);
      const double cq = cc[q];
      const cplx sq = ss[q];
      Rm[(int64_t)jj * M + q] = cadd(cscale(carry, cq), cmul(sq, b));
      carry = cadd(cmul(cmk(-sq.x, sq.y), carry), cscale(b, cq));
    }
    double cn;
    cplx sn, rr;
    givens(carry, hcol[jj + 1], cn, sn, rr);
    cc[jj] = cn;
    ss[jj] = sn;
    Rm[(int64_t)jj * M + jj] = rr;
    const cplx gj = yy[jj];
    yy[jj] = cscale(gj, cn);
    yy[jj + 1] = cmul(cmk(-sn.x, sn.y), gj);
  }
  for (int i = J - 1; i >= 0; --i) {
    cplx acc = yy[i];
    for (int m = i + 1; m < J; ++m) acc = cfms(Rm[(int64_t)m * M + i], yy[m], acc);
    const cplx d = Rm[(int64_t)i * M + i];
    yy[i] = (d.x == 0.0 && d.y == 0.0) ? cmk(0, 0) : cdiv(acc, d);
  }
}

__global__ void zcombine_kernel(KrylovDev K, int k, const cplx* wts, int nshift, double odd,
                                const cplx* y, cplx* z) {
  const int c = blockIdx.x;
  const int J = K.jc[c];
  const int M = K.m_max;
  // the odd-p term needs v_0 even when no Arnoldi step was taken
  const int Jz = (K.beta[c] > 0.0) ? max(J, 1) : 0;
  for (int i = threadIdx.x; i < Jz; i += blockDim.x) {
    cplx acc = cmk(0, 0);
    if (i < J)
      for (int l = 0; l < nshift; ++l)
        acc = cfms(wts[l], y[((int64_t)c * nshift + l) * (M + 1) + i], acc);
    if (i == 0) acc = cadd(acc, cmk(odd * K.beta[c], 0.0));
    z[(int64_t)c * (M + 1) + i] = acc;
  }
}

__global__ void vz_kernel(KrylovDev K, const cplx* z, cplx* U, int64_t ldu) {
  const int c = blockIdx.y;
  const int M = K.m_max;
  const int J = (K.beta[c] > 0.0) ? max(K.jc[c], 1) : 0;
  __shared__ cplx zs[1024];
  for (int i = threadIdx.x; i < J; i += blockDim.x) zs[i] = z[(int64_t)c * (M + 1) + i];
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= K.n) return;
  const cplx* Vc = K.V + (int64_t)c * (M + 1) * K.n;
  cplx acc = cmk(0, 0);
  for (int i = 0; i < J; ++i) acc = cfma(Vc[(int64_t)i * K.n + r], zs[i], acc);
  U[(int64_t)c * ldu + r] = acc;
}

void launch_krylov_combine(const KrylovDev& K, int k, const cplx* d_shifts, const cplx* d_wts,
                           int nshift, double odd, cplx* Rscratch, cplx* zbuf, cplx* U,
                           int64_t ldu, cudaStream_t s) {
  // zbuf layout: [rot_c k*nshift*M doubles as cplx][rot_s][y k*nshift*(M+1)][z k*(M+1)]
  const int M = K.m_max;
  cplx* rot_c = zbuf;
  cplx* rot_s = rot_c + (int64_t)k * nshift * M;
  cplx* y = rot_s + (int64_t)k * nshift * M;
  cplx* z = y + (int64_t)k * nshift * (M + 1);
  const int tot = k * nshift;
  if (nshift > 0)
    ls_solve_kernel<<<(tot + 63) / 64, 64, 0, s>>>(K, k, d_shifts, nshift, (double*)rot_c, rot_s,
                                                  Rscratch, y); ie_count_launch();
  zcombine_kernel<<<k, 128, 0, s>>>(K, k, d_wts, nshift, odd, y, z); ie_count_launch();
  vz_kernel<<<dim3((unsigned)((K.n + 255) / 256), k), 256, 0, s>>>(K, z, U, ldu); ie_count_launch();
}

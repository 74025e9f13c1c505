// Band kernels of the inner operator G (Sec. 3.2, Eq. linearsolve2):
//   assembly of K_i = p_i B - A (Alg. 1) into LAPACK band storage,
//   batched band LU with partial pivoting over all q poles in one cooperative launch,
//   the DIA SpMV with A and B, the pole sums, and the complex64 factor copy and FP64
//   residuals of the mixed-precision path (the triangular solves are in ie_solve.cu).
#include <cooperative_groups.h>
#include <cstdio>

#include <atomic>

#include <cstdlib>

#include "ie_internal.cuh"

static std::atomic<int64_t> g_launches{0};
void ie_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
int64_t ie_launch_count() { return g_launches.load(std::memory_order_relaxed); }

// ----------------------------------------------------------------------------------------------
// SpMV: Y = (aA A + aB B) X on a block, DIA storage M[i, i+off_d] = dia[d*n + i].
__global__ void spmv_dia_kernel(DiaDev P, cplx aA, cplx aB, int useA, int useB, const cplx* X,
                                int64_t ldx, const int64_t* xoff, cplx* Y, int64_t ldy) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= P.n) return;
  const cplx* xc = xoff ? X + xoff[c] : X + (int64_t)c * ldx;
  cplx acc = cmk(0.0, 0.0);
  for (int d = 0; d < P.ndiag; ++d) {
    const int64_t j = i + P.off[d];
    if (j < 0 || j >= P.n) continue;
    cplx m = cmk(0.0, 0.0);
    if (useA) m = cmul(aA, P.A[(int64_t)d * P.n + i]);
    if (useB) m = cfma(aB, P.B[(int64_t)d * P.n + i], m);
    acc = cfma(m, xc[j], acc);
  }
  Y[(int64_t)c * ldy + i] = acc;
}

void launch_spmv(const DiaDev& P, cplx aA, cplx aB, const cplx* X, int64_t ldx,
                 const int64_t* xoff, int k, cplx* Y, int64_t ldy, cudaStream_t s) {
  if (k <= 0 || P.n <= 0) return;
  const int useA = (aA.x != 0.0 || aA.y != 0.0), useB = (aB.x != 0.0 || aB.y != 0.0);
  dim3 grid((unsigned)((P.n + 255) / 256), (unsigned)k);
  spmv_dia_kernel<<<grid, 256, 0, s>>>(P, aA, aB, useA, useB, X, ldx, xoff, Y, ldy); ie_count_launch();
}

// ----------------------------------------------------------------------------------------------
// Assembly: AB[i][j*ldab + t] = K_i(j + t - kv, j) for t in [kl, ldab), zero fill rows t < kl,
// zero outside the matrix and for padding columns j >= n. kv = 2 kl.
__device__ __forceinline__ void put_c(float2* p, cplx v) { *p = make_float2((float)v.x, (float)v.y); }
__device__ __forceinline__ void put_c(cplx* p, cplx v) { *p = v; }

// K_i entries are formed in complex128 and stored in the factor precision (complex64 for the
// mixed-precision path: the rounding of K_i itself, the first error the refinement removes).
template <typename OT>
__global__ void assemble_kernel(DiaDev P, const cplx* poles, int kl, int ldab, int64_t n_pad,
                                OT* AB) {
  const int pole = blockIdx.y;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_pad * ldab) return;
  const int64_t j = idx / ldab;
  const int t = (int)(idx - j * ldab);
  const int kv = 2 * kl;
  cplx v = cmk(0.0, 0.0);
  if (j < P.n && t >= kl) {
    const int64_t r = j + t - kv;
    if (r >= 0 && r < P.n) {
      const int64_t off = j - r;   // column - row
      const cplx p = poles[pole];
      for (int d = 0; d < P.ndiag; ++d) {
        if (P.off[d] == off) {
          const cplx a = P.A[(int64_t)d * P.n + r];
          const cplx b = P.B[(int64_t)d * P.n + r];
          v = csub(cmul(p, b), a);       // K = p B - A
        }
      }
    }
  }
  put_c(&AB[(int64_t)pole * n_pad * ldab + idx], v);
}

template <typename OT>
static void assemble_t(const DiaDev& P, const cplx* d_poles, int q, int kl, int ldab,
                       int64_t n_pad, OT* AB, cudaStream_t s) {
  const int64_t tot = n_pad * ldab;
  dim3 grid((unsigned)((tot + 255) / 256), (unsigned)q);
  assemble_kernel<OT><<<grid, 256, 0, s>>>(P, d_poles, kl, ldab, n_pad, AB); ie_count_launch();
}
void launch_assemble(const DiaDev& P, const cplx* d_poles, int q, int kl, int ldab,
                     int64_t n_pad, cplx* AB, cudaStream_t s) {
  assemble_t(P, d_poles, q, kl, ldab, n_pad, AB, s);
}
void launch_assemble(const DiaDev& P, const cplx* d_poles, int q, int kl, int ldab,
                     int64_t n_pad, float2* AB, cudaStream_t s) {
  assemble_t(P, d_poles, q, kl, ldab, n_pad, AB, s);
}

// ----------------------------------------------------------------------------------------------
// ||M||_1 = max_j sum_d |M(j - off_d, j)| = max_j sum_d |dia[d][j - off_d]|.
__global__ void norm1_kernel(DiaDev P, int which, unsigned long long* out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double s = 0.0;
  if (j < P.n) {
    const cplx* M = which ? P.B : P.A;
    for (int d = 0; d < P.ndiag; ++d) {
      const int64_t r = j - P.off[d];
      if (r >= 0 && r < P.n) s += cabsv(M[(int64_t)d * P.n + r]);
    }
  }
  for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_xor_sync(0xffffffffu, s, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(s));
}

void launch_norm1_cols(const DiaDev& P, int which, double* d_out, double* /*scratch*/,
                       cudaStream_t s) {
  cudaMemsetAsync(d_out, 0, sizeof(double), s);
  norm1_kernel<<<(unsigned)((P.n + 255) / 256), 256, 0, s>>>(P, which,
                                                               (unsigned long long*)d_out); ie_count_launch();
}

// ----------------------------------------------------------------------------------------------
// Batched band LU with partial pivoting (LAPACK zgbtf2 semantics, 0-based):
// for each column j: pivot row j+tp = argmax_t |re|+|im| of column j rows j..j+kl (first max);
// ju = max(ju, min(j + ku + tp, n-1)); swap rows j and j+tp in columns j..ju; multipliers
// l_t = a(j+t, j) / pivot; rank-1 update of rows j+1..j+kl in columns j+1..ju.
// Grid = q poles x P CTAs; CTA b owns the columns l with l % P == b, and only it reads or
// writes them. Look-ahead: at step j the owner of column j+1 applies step j to that column
// first, finds its pivot and multipliers, writes its final entries (U(j+1,j+1), L, piv,
// 1/pivot) and publishes (pivot offset, multipliers) for step j+1 in a per-pole ring slot,
// then sets the slot's flag with release semantics. Every other CTA of the pole waits only on
// that flag (bounded, abort-aware) before applying step j+1 to its own columns, so no barrier
// spans the pole and the owner's next pivot overlaps the other CTAs' updates. A CTA can run
// at most P steps ahead of another (each CTA owns one column in any P consecutive ones, and
// its pivot gates that step), so R >= P + 2 ring slots are never overwritten while read.

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *(const volatile int*)p;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Waits (thread 0 of the CTA) until flag == want; false on timeout or abort.
__device__ bool lu_wait_flag(const unsigned* flag, unsigned want, int* status) {
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    int ok = 1;
    if (ld_acquire_u32(flag) != want) {
      const unsigned long long t0 = ie_globaltimer();
      unsigned it = 0;
      while (ld_acquire_u32(flag) != want) {
        if ((++it & 15u) == 0) {
          if (ld_volatile_i32(status + ST_ABORT)) { ok = 0; break; }
          if (ie_globaltimer() - t0 > IE_WAIT_NS) {
            atomicExch(status + ST_TIMEOUT, 1);
            atomicExch(status + ST_ABORT, 1);
            ok = 0;
            break;
          }
        }
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Element arithmetic of the band LU for complex128 and complex64 (FP32 accumulation).
__device__ __forceinline__ double lu_abs1(cplx a) { return fabs(a.x) + fabs(a.y); }
__device__ __forceinline__ float lu_abs1(float2 a) { return fabsf(a.x) + fabsf(a.y); }
__device__ __forceinline__ cplx lu_mul(cplx a, cplx b) { return cmul(a, b); }
__device__ __forceinline__ float2 lu_mul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ cplx lu_fms(cplx a, cplx b, cplx c) { return cfms(a, b, c); }
__device__ __forceinline__ float2 lu_fms(float2 a, float2 b, float2 c) {   // c - a*b
  return make_float2(fmaf(-a.x, b.x, fmaf(a.y, b.y, c.x)), fmaf(-a.x, b.y, fmaf(-a.y, b.x, c.y)));
}
__device__ __forceinline__ cplx lu_rcp(cplx b) { return crcp(b); }
// 1/b by Smith's algorithm (R. L. Smith, CACM 5(8), 1962), in FP32
__device__ __forceinline__ float2 lu_rcp(float2 b) {
  if (fabsf(b.x) >= fabsf(b.y)) {
    const float r = b.y / b.x, d = b.x + b.y * r;
    return make_float2(1.0f / d, -r / d);
  }
  const float r = b.x / b.y, d = b.y + b.x * r;
  return make_float2(r / d, -1.0f / d);
}
template <typename CT> __device__ __forceinline__ CT lu_zero() { return CT{}; }

template <typename CT>
__global__ void __launch_bounds__(512) band_lu_kernel(int64_t n, int kl, int ldab, int64_t n_pad,
                                                      CT* AB, int* piv, CT* dinv,
                                                      CT* ring, int* ring_tp,
                                                      unsigned* ring_flag, int R, int* status,
                                                      int P, int nown_max, int64_t skip_publish) {
  using RT = decltype(lu_abs1(CT{}));
  const int pole = blockIdx.x / P, b = blockIdx.x % P;
  const int T = blockDim.x, tid = threadIdx.x;
  const int kv = 2 * kl;
  CT* A = AB + (int64_t)pole * n_pad * ldab;
  int* pv_out = piv + (int64_t)pole * n_pad;
  CT* di_out = dinv + (int64_t)pole * n_pad;
  CT* rmul = ring + (int64_t)pole * R * (kl + 1);
  int* rtp = ring_tp + (int64_t)pole * R;
  unsigned* rflag = ring_flag + (int64_t)pole * R;
  extern __shared__ __align__(16) unsigned char lu_sm_raw[];
  CT* mult = (CT*)lu_sm_raw;         // kl+1: multipliers of the current step
  CT* col = mult + (kl + 1);         // kl+1: pivot column of the next step (owner)
  CT* urow = col + (kl + 1);         // nown_max
  CT* arow = urow + nown_max;        // nown_max
  __shared__ RT red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_tp;

  // pivot search, multipliers, final column entries and publication of step jc (owner of
  // column jc only); column jc holds all updates of steps < jc in global memory
  // col[0..pre) already holds rows jc..jc+pre-1 of the column (the look-ahead update)
  auto pivot_publish = [&](int64_t jc, int pre, int jcr /* jc % R */) {
    const int nr = (int)((n - 1 - jc) < (int64_t)kl ? (n - 1 - jc) : (int64_t)kl);
    CT* cj = A + jc * ldab + kv;
    RT best = -1;
    int bi = 0;
    for (int t = tid; t <= nr; t += T) {
      const CT v = (t < pre) ? col[t] : __ldcg(cj + t);
      col[t] = v;
      const RT a = lu_abs1(v);
      if (a > best) { best = a; bi = t; }
    }
    for (int o = 16; o > 0; o >>= 1) {   // argmax, first index on ties
      const RT ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
      RT bb = red_v[0];
      int ii = red_i[0];
      for (int w = 1; w < (T + 31) / 32; ++w)
        if (red_v[w] > bb || (red_v[w] == bb && red_i[w] < ii)) { bb = red_v[w]; ii = red_i[w]; }
      s_tp = ii;
    }
    __syncthreads();
    const int tp = s_tp;
    const CT pv = col[tp];
    const bool zero = (pv.x == 0 && pv.y == 0);
    const CT rcp = zero ? lu_zero<CT>() : lu_rcp(pv);
    CT* slot = rmul + (int64_t)jcr * (kl + 1);
    for (int t = tid; t <= nr; t += T) {
      if (t == 0) {
        cj[0] = pv;
      } else {
        const CT m = zero ? lu_zero<CT>() : lu_mul((t == tp) ? col[0] : col[t], rcp);
        cj[t] = m;
        slot[t] = m;
      }
    }
    if (tid == 0) {
      if (zero) atomicMax(status + ST_SINGULAR, 1);
      pv_out[jc] = (int)(jc + tp);
      di_out[jc] = rcp;
      rtp[jcr] = tp;
    }
    __syncthreads();
    if (tid == 0 && jc != skip_publish) {   // skip_publish: failure test hook (normally -1)
      __threadfence();
      st_release_u32(rflag + jcr, (unsigned)(jc + 1));
    }
  };

  if (n > 0 && b == 0) pivot_publish(0, 0, 0);
  int64_t ju = 0;
  // jr = j % R and jp = j % P as running counters (no 64-bit division per step)
  int jr = 0, jp = 0;
  for (int64_t j = 0; j < n; ++j, jr = (jr + 1 == R) ? 0 : jr + 1, jp = (jp + 1 == P) ? 0 : jp + 1) {
    const int jr1 = (jr + 1 == R) ? 0 : jr + 1, jp1 = (jp + 1 == P) ? 0 : jp + 1;
    // (a) step j's pivot offset and multipliers, published by the owner of column j
    if (!lu_wait_flag(rflag + jr, (unsigned)(j + 1), status)) return;
    const int nrows = (int)((n - 1 - j) < (int64_t)kl ? (n - 1 - j) : (int64_t)kl);
    const CT* slot = rmul + (int64_t)jr * (kl + 1);
    for (int t = 1 + tid; t <= nrows; t += T) mult[t] = __ldcg(slot + t);
    const int tp = __ldcg(rtp + jr);
    { const int64_t cand = (j + kl + tp < n - 1) ? (j + kl + tp) : (n - 1); if (cand > ju) ju = cand; }
    __syncthreads();
    // (b) look-ahead: the owner of column j+1 applies step j to it, then publishes step j+1
    const bool own_next = (j + 1 < n) && (jp1 == b);
    if (own_next) {
      int pre = 0;
      if (j + 1 <= ju && nrows > 0) {
        CT* cl = A + (j + 1) * ldab + kv - 1;        // row j of column j+1
        const CT u = __ldcg(cl + tp), a0 = __ldcg(cl);
        __syncthreads();                             // rows j and j+tp read before rewritten
        for (int t = tid; t <= nrows; t += T) {
          if (t == 0) {
            cl[0] = u;
          } else {
            const CT nv = lu_fms(mult[t], u, (t == tp) ? a0 : __ldcg(cl + t));
            cl[t] = nv;
            col[t - 1] = nv;                         // row j+t = row (j+1)+(t-1) of the column
          }
        }
        pre = nrows;
        __syncthreads();
      }
      pivot_publish(j + 1, pre, jr1);
    }
    // (c) swap + rank-1 update of the other owned columns l in (j, ju], l % P == b
    const int64_t jn = own_next ? j + 2 : j + 1;    // column j+1 is done when owned here
    const int jnp = own_next ? ((jp1 + 1 == P) ? 0 : jp1 + 1) : jp1;   // jn % P
    const int64_t l0 = jn + ((b - jnp < 0) ? b - jnp + P : b - jnp);
    const int nown = (l0 <= ju && nrows >= 0) ? (int)(ju - l0) / P + 1 : 0;
    for (int idx = tid; idx < nown; idx += T) {
      const int64_t l = l0 + (int64_t)idx * P;
      const CT* cl = A + l * ldab + kv - (l - j);     // row j of column l
      urow[idx] = __ldcg(cl + tp);
      arow[idx] = __ldcg(cl);
    }
    __syncthreads();
    if (nown > 0 && nrows > 0) {
      // rank-1 update, LU_BATCH independent loads in flight per thread before the stores
      constexpr int LU_BATCH = 8;
      const int tot = nrows * nown;
      for (int it0 = tid; it0 < tot; it0 += T * LU_BATCH) {
        CT val[LU_BATCH];
        CT* dst[LU_BATCH];
        int tt[LU_BATCH], ii[LU_BATCH];
#pragma unroll
        for (int u = 0; u < LU_BATCH; ++u) {
          const int it = it0 + u * T;
          ii[u] = -1;
          if (it < tot) {
            const int idx = it / nrows;
            const int t = 1 + (it - idx * nrows);
            const int64_t l = l0 + (int64_t)idx * P;
            dst[u] = A + l * ldab + kv - (l - j) + t;
            tt[u] = t;
            ii[u] = idx;
            val[u] = (t == tp) ? arow[idx] : __ldcg(dst[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < LU_BATCH; ++u)
          if (ii[u] >= 0) *dst[u] = lu_fms(mult[tt[u]], urow[ii[u]], val[u]);
      }
    }
    for (int idx = tid; idx < nown; idx += T) {
      const int64_t l = l0 + (int64_t)idx * P;
      A[l * ldab + kv - (l - j)] = urow[idx];
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------------------------
// Blocked form of the same factorisation: panels of LNB = 16 columns. CTA b of a pole owns the
// column blocks K with K % P == b. The owner of panel J factors it on a register tile (rows
// J*LNB .. J*LNB + LNB - 1 + kl, the panel's LNB columns) with barriers of its own CTA only,
// and publishes the panel's multipliers, pivot offsets and column extent ju in a per-pole ring
// slot (release flag, as above). Every CTA then applies panel J to each of its blocks in reach
// (columns up to ju) on a register tile of the same rows: the panel's LNB steps (row swap,
// then rank-1 elimination) in gbtf2's order, one barrier per step; a block is loaded from the
// band storage once per panel and written back once. Look-ahead: the owner of block J+1
// applies panel J to it first, factors it and publishes panel J+1 before its other blocks.
// Every element receives exactly the operations of band_lu_kernel in the same order (steps
// that gbtf2 skips for a column beyond ju act on exact zeros and leave it unchanged), so the
// factors are identical; only the synchronisation differs: one flag per 16 columns instead of
// one per column, and the column block stays on chip for the 16 steps.
constexpr int LNB = 16;        // panel width
constexpr int LTR = 128;       // row lanes of a tile (threads tid & 127)
constexpr int LRPT = 5;        // rows per thread at most: tiles up to 640 rows (kl <= 624)

template <typename CT, int RPT>
struct LuTile {
  CT v[RPT][LNB / 4];
};

// RPT: tile rows per thread (3 for tiles of <= 384 rows, 5 up to 640)
template <typename CT, int RPT>
__global__ void __launch_bounds__(512, 1) band_lu_blocked_kernel(
    int64_t n, int kl, int ldab, int64_t n_pad, CT* AB, int* piv, CT* dinv, CT* ring,
    int* ring_tp, unsigned* ring_flag, int R, int* status, int P, int64_t skip_publish) {
  using RT = decltype(lu_abs1(CT{}));
  const int pole = blockIdx.x / P, b = blockIdx.x % P;
  const int tid = threadIdx.x, tx = tid & (LTR - 1), ty = tid >> 7;   // 4 column groups
  const int kv = 2 * kl;
  const int RTL = LNB + kl;                 // tile rows
  const int64_t npan = (n + LNB - 1) / LNB;
  CT* A = AB + (int64_t)pole * n_pad * ldab;
  int* pv_out = piv + (int64_t)pole * n_pad;
  CT* di_out = dinv + (int64_t)pole * n_pad;
  // ring slot: LNB columns of kl multipliers, then (in ring_tp) LNB pivot offsets + ju
  CT* rmul = ring + (int64_t)pole * R * LNB * kl;
  int* rtp = ring_tp + (int64_t)pole * R * (LNB + 1);
  unsigned* rflag = ring_flag + (int64_t)pole * R;
  extern __shared__ __align__(16) unsigned char lu_sm_raw[];
  CT* msm = (CT*)lu_sm_raw;                 // [LNB][kl]: staged multipliers of the applied panel
  CT* ubuf = msm + (size_t)LNB * kl;        // [2][LNB]: pivot row after the swap
  CT* wbuf = ubuf + 2 * LNB;                // [2][LNB]: old row j (goes to the pivot row)
  CT* mcol = wbuf + 2 * LNB;                // [2][RTL]: multipliers of the current factor step
  __shared__ int s_tp[LNB + 1];
  __shared__ RT red_v[4];
  __shared__ int red_i[4];

  auto stor = [&](int64_t r, int64_t c) -> bool {   // (r, c) inside the band storage
    return c < n && r < n && r >= c - kv && r <= c + kl;
  };
  auto load_tile = [&](int64_t J, int64_t K, LuTile<CT, RPT>& t) {
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int rr = tx + i * LTR;
      const int64_t r = J * LNB + rr;
#pragma unroll
      for (int q = 0; q < LNB / 4; ++q) {
        const int64_t c = K * LNB + ty * (LNB / 4) + q;
        t.v[i][q] = (rr < RTL && stor(r, c)) ? A[c * ldab + kv + (r - c)] : lu_zero<CT>();
      }
    }
  };
  auto store_tile = [&](int64_t J, int64_t K, const LuTile<CT, RPT>& t) {
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int rr = tx + i * LTR;
      const int64_t r = J * LNB + rr;
#pragma unroll
      for (int q = 0; q < LNB / 4; ++q) {
        const int64_t c = K * LNB + ty * (LNB / 4) + q;
        if (rr < RTL && stor(r, c)) A[c * ldab + kv + (r - c)] = t.v[i][q];
      }
    }
  };
  // steps of panel J (multipliers in msm, offsets in s_tp) on block K's tile
  auto apply_panel = [&](int64_t J, LuTile<CT, RPT>& t) {
    const int nst = (int)((n - J * LNB) < LNB ? (n - J * LNB) : LNB);
    for (int jj = 0; jj < nst; ++jj) {
      const int tp = s_tp[jj];
      const int buf = jj & 1;
      // rows j = jj and p = jj + tp of the tile publish their values
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int rr = tx + i * LTR;
#pragma unroll
        for (int q = 0; q < LNB / 4; ++q) {
          if (rr == jj) wbuf[buf * LNB + ty * (LNB / 4) + q] = t.v[i][q];
          if (rr == jj + tp) ubuf[buf * LNB + ty * (LNB / 4) + q] = t.v[i][q];
        }
      }
      __syncthreads();
      const CT* m = msm + (size_t)jj * kl;   // m[t - 1]: multiplier of row j + t
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int rr = tx + i * LTR;
        const int d = rr - jj;
#pragma unroll
        for (int q = 0; q < LNB / 4; ++q) {
          const int cc = ty * (LNB / 4) + q;
          const CT u = ubuf[buf * LNB + cc];
          if (d == 0) {
            t.v[i][q] = u;
          } else if (d > 0 && d <= kl) {
            const CT base = (d == tp) ? wbuf[buf * LNB + cc] : t.v[i][q];
            t.v[i][q] = lu_fms(m[d - 1], u, base);
          }
        }
      }
    }
    __syncthreads();
  };
  // factor panel J on its tile: pivot search, swap (panel columns >= jj), multipliers,
  // elimination of the panel columns > jj; results in the tile; piv/dinv written
  // ju_init: gbtf2's running column extent after the previous panel (ju never decreases)
  auto factor_panel = [&](int64_t J, LuTile<CT, RPT>& t, int64_t ju_init, int* ju_out) {
    const int nst = (int)((n - J * LNB) < LNB ? (n - J * LNB) : LNB);
    int64_t ju = ju_init;
    for (int jj = 0; jj < nst; ++jj) {
      const int64_t j = J * LNB + jj;
      const int nr = (int)((n - 1 - j) < (int64_t)kl ? (n - 1 - j) : (int64_t)kl);
      const int buf = jj & 1;
      // pivot search over column jj, tile rows jj..jj+nr (first max of |re| + |im|)
      const int gq = jj / (LNB / 4), qq = jj - gq * (LNB / 4);
      if (ty == gq) {
        RT best = -1;
        int bi = 0;
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const int rr = tx + i * LTR;
          const int d = rr - jj;
          if (d >= 0 && d <= nr) {
            RT a_ = 0;
#pragma unroll
            for (int q = 0; q < LNB / 4; ++q)
              if (q == qq) a_ = lu_abs1(t.v[i][q]);
            if (a_ > best || (a_ == best && d < bi)) { best = a_; bi = d; }
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          const RT ob = __shfl_xor_sync(0xffffffffu, best, o);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
          if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
        }
        if ((tx & 31) == 0) { red_v[tx >> 5] = best; red_i[tx >> 5] = bi; }
      }
      __syncthreads();
      if (tid == 0) {
        RT bb = red_v[0];
        int ii = red_i[0];
        for (int w = 1; w < 4; ++w)
          if (red_v[w] > bb || (red_v[w] == bb && red_i[w] < ii)) { bb = red_v[w]; ii = red_i[w]; }
        s_tp[jj] = ii;
      }
      __syncthreads();
      const int tp = s_tp[jj];
      { const int64_t cand = (j + kl + tp < n - 1) ? (j + kl + tp) : (n - 1); if (cand > ju) ju = cand; }
      // rows j and p publish their values of the panel columns >= jj
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int rr = tx + i * LTR;
#pragma unroll
        for (int q = 0; q < LNB / 4; ++q) {
          const int cc = ty * (LNB / 4) + q;
          if (cc < jj) continue;
          if (rr == jj) wbuf[buf * LNB + cc] = t.v[i][q];
          if (rr == jj + tp) ubuf[buf * LNB + cc] = t.v[i][q];
        }
      }
      __syncthreads();
      const CT pvv = ubuf[buf * LNB + jj];
      const bool zero = (pvv.x == 0 && pvv.y == 0);
      const CT rcp = zero ? lu_zero<CT>() : lu_rcp(pvv);
      // column jj: the swap and the multipliers (kept in the tile as L, and in mcol)
      if (ty == gq) {
#pragma unroll
        for (int i = 0; i < RPT; ++i) {
          const int rr = tx + i * LTR;
          const int d = rr - jj;
#pragma unroll
          for (int q = 0; q < LNB / 4; ++q) {
            if (q != qq) continue;
            if (d == 0) {
              t.v[i][q] = pvv;
            } else if (d > 0 && d <= nr) {
              const CT m = zero ? lu_zero<CT>() : lu_mul((d == tp) ? wbuf[buf * LNB + jj] : t.v[i][q], rcp);
              t.v[i][q] = m;
              mcol[buf * RTL + rr] = m;
            }
          }
        }
      }
      if (tid == 0) {
        if (zero) atomicMax(status + ST_SINGULAR, 1);
        pv_out[j] = (int)(j + tp);
        di_out[j] = rcp;
      }
      __syncthreads();
      // elimination of the panel columns > jj
#pragma unroll
      for (int i = 0; i < RPT; ++i) {
        const int rr = tx + i * LTR;
        const int d = rr - jj;
#pragma unroll
        for (int q = 0; q < LNB / 4; ++q) {
          const int cc = ty * (LNB / 4) + q;
          if (cc <= jj) continue;
          const CT u = ubuf[buf * LNB + cc];
          if (d == 0) {
            t.v[i][q] = u;
          } else if (d > 0 && d <= nr) {
            const CT base = (d == tp) ? wbuf[buf * LNB + cc] : t.v[i][q];
            t.v[i][q] = lu_fms(mcol[buf * RTL + rr], u, base);
          }
        }
      }
    }
    __syncthreads();
    *ju_out = (int)ju;
  };
  // publish panel J: multipliers of each column (from the tile), offsets, ju; then the flag
  auto publish = [&](int64_t J, const LuTile<CT, RPT>& t, int ju) {
    const int nst = (int)((n - J * LNB) < LNB ? (n - J * LNB) : LNB);
    CT* slot = rmul + (J % R) * LNB * kl;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int rr = tx + i * LTR;
#pragma unroll
      for (int q = 0; q < LNB / 4; ++q) {
        const int cc = ty * (LNB / 4) + q;
        const int d = rr - cc;
        if (cc < nst && d >= 1 && d <= kl) slot[(size_t)cc * kl + d - 1] = t.v[i][q];
      }
    }
    if (tid < LNB) rtp[(J % R) * (LNB + 1) + tid] = s_tp[tid];
    if (tid == 0) rtp[(J % R) * (LNB + 1) + LNB] = ju;
    __syncthreads();
    if (tid == 0 && J != skip_publish) {   // skip_publish: failure test hook (normally -1)
      __threadfence();
      st_release_u32(rflag + (J % R), (unsigned)(J + 1));
    }
  };
  auto owner = [&](int64_t K) { return (int)(K % P); };

  LuTile<CT, RPT> tile;
  if (npan > 0 && owner(0) == b) {
    int ju;
    load_tile(0, 0, tile);
    factor_panel(0, tile, 0, &ju);
    store_tile(0, 0, tile);
    publish(0, tile, ju);
  }
  int Jr = 0;   // J % R, running
  for (int64_t J = 0; J < npan; ++J, Jr = (Jr + 1 == R) ? 0 : Jr + 1) {
    if (!lu_wait_flag(rflag + Jr, (unsigned)(J + 1), status)) return;
    // stage panel J: multipliers, offsets, column extent
    const CT* slot = rmul + (int64_t)Jr * LNB * kl;
    for (int e = tid; e < LNB * kl; e += blockDim.x) msm[e] = __ldcg(slot + e);
    if (tid <= LNB) s_tp[tid] = __ldcg(rtp + Jr * (LNB + 1) + tid);
    __syncthreads();
    const int64_t ju = s_tp[LNB];
    const int64_t kmax = ju / LNB < npan - 1 ? ju / LNB : npan - 1;
    // look-ahead: block J+1 first, then its factorisation and publication
    const bool own_next = J + 1 < npan && owner(J + 1) == b;
    if (own_next) {
      int jun;
      load_tile(J, J + 1, tile);
      apply_panel(J, tile);
      store_tile(J, J + 1, tile);
      __syncthreads();
      // panel J+1's tile starts one panel lower: reload it from the band storage
      load_tile(J + 1, J + 1, tile);
      factor_panel(J + 1, tile, ju, &jun);
      store_tile(J + 1, J + 1, tile);
      publish(J + 1, tile, jun);
      // the staged panel J was overwritten by s_tp of panel J+1: restore the offsets
      if (tid <= LNB) s_tp[tid] = __ldcg(rtp + Jr * (LNB + 1) + tid);
      __syncthreads();
    }
    // this CTA's blocks K in (J + own_next, kmax]: the first by one modulo, then every P-th
    const int64_t K0 = J + 1 + (own_next ? 1 : 0);
    const int dk = (int)(((int64_t)b - K0 % P + P) % P);
    for (int64_t K = K0 + dk; K <= kmax; K += P) {
      load_tile(J, K, tile);
      apply_panel(J, tile);
      store_tile(J, K, tile);
    }
    __syncthreads();
  }
}

// Ring storage a pole needs: multipliers (elements of the factor type) and offsets (ints).
size_t band_lu_ring_elems(int q, int kl) {
  const size_t R = (size_t)band_lu_ring_slots(q);
  return (size_t)q * R * (size_t)LNB * (size_t)(kl + 1);
}
size_t band_lu_ring_ints(int q) { return (size_t)q * (size_t)band_lu_ring_slots(q) * (LNB + 1); }

int band_lu_ring_slots(int q) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int pmax = sms / (q > 0 ? q : 1);
  return 2 * (pmax > 1 ? pmax : 1) + 2;
}

// IE_LU_BLOCKED=0 in the environment selects the column-by-column kernel (the same factors).
static bool lu_blocked_enabled() {
  static const bool on = [] {
    const char* e = getenv("IE_LU_BLOCKED");
    return !(e && e[0] == '0');
  }();
  return on;
}

template <typename CT>
static cudaError_t band_lu_blocked_t(int q, int64_t n, int kl, int ldab, int64_t n_pad, CT* AB,
                                     int* piv, CT* dinv, CT* ring, int* ring_tp,
                                     unsigned* ring_flag, int R, int* status, cudaStream_t s,
                                     int* ctas_per_pole) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int kv = 2 * kl;
  int P = sms / q;
  if (P > kv / LNB + 2) P = kv / LNB + 2;   // blocks one panel can reach, plus the next panel
  if (P > R - 2) P = R - 2;                 // ring slots outlive the CTAs' spread (see above)
  if (P < 1) return cudaErrorInvalidValue;
  const size_t smem = ((size_t)LNB * kl + 4 * LNB + 2 * (LNB + kl)) * sizeof(CT);
  auto kfn = (LNB + kl <= 3 * LTR) ? band_lu_blocked_kernel<CT, 3> : band_lu_blocked_kernel<CT, 5>;
  ie_smem_optin((const void*)kfn);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 512, smem);
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  while ((int64_t)P * q > (int64_t)per_sm * sms && P > 1) --P;
  if (ctas_per_pole) *ctas_per_pole = P;
  cudaMemsetAsync(ring_flag, 0, sizeof(unsigned) * (size_t)R * q, s);
  // Failure test hook: IE_TEST_SKIP_PUBLISH=J makes the owner of panel J never set its flag
  // (every wait for that panel runs out after IE_WAIT_NS; ie_create reports IE_ERR_TIMEOUT).
  int64_t skip_publish = -1;
  if (const char* e = getenv("IE_TEST_SKIP_PUBLISH")) skip_publish = atoll(e);
  void* args[] = {&n, &kl, &ldab, &n_pad, &AB, &piv, &dinv, &ring, &ring_tp, &ring_flag, &R,
                  &status, &P, &skip_publish};
  ie_count_launch();
  return cudaLaunchCooperativeKernel((void*)kfn, dim3(q * P), dim3(512), args, smem, s);
}

template <typename CT>
static cudaError_t band_lu_t(int q, int64_t n, int kl, int ldab, int64_t n_pad, CT* AB, int* piv,
                             CT* dinv, CT* ring, int* ring_tp, unsigned* ring_flag, int R,
                             int* status, cudaStream_t s, int* ctas_per_pole) {
  // complex64: the blocked kernel (C2 236 ms against 413 ms column by column, C4 1.9 s
  // against 4.2 s). complex128: the column-by-column kernel, which the FP64 units bound (the
  // blocked one measured 1.03 s against 0.79 s at C2: the same FP64 work, spread less evenly)
  if constexpr (sizeof(CT) == sizeof(float2)) {
    if (lu_blocked_enabled() && LNB + kl <= LTR * LRPT)
      return band_lu_blocked_t(q, n, kl, ldab, n_pad, AB, piv, dinv, ring, ring_tp, ring_flag, R,
                               status, s, ctas_per_pole);
  }
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int kv = 2 * kl;
  int P = sms / q;
  if (P < 1) P = 1;
  if (P > kv) P = kv;
  // a ring slot is rewritten R steps after its last reader could still need it: CTAs are at
  // most P + 1 steps apart (the slowest one publishes the pivot of one of every P columns)
  if (P > R - 2) P = R - 2;
  if (P < 1) return cudaErrorInvalidValue;
  int nown_max = (kv + P - 1) / P + 1;
  size_t smem = (size_t)(2 * (kl + 1) + 2 * nown_max) * sizeof(CT);
  auto kfn = band_lu_kernel<CT>;
  if (smem > 48 * 1024) ie_smem_optin((const void*)kfn);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 512, smem);
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  while ((int64_t)P * q > (int64_t)per_sm * sms && P > 1) {
    --P;
    nown_max = (kv + P - 1) / P + 1;
  }
  smem = (size_t)(2 * (kl + 1) + 2 * nown_max) * sizeof(CT);
  if (ctas_per_pole) *ctas_per_pole = P;
  cudaMemsetAsync(ring_flag, 0, sizeof(unsigned) * (size_t)R * q, s);
  // Failure test hook: IE_TEST_SKIP_PUBLISH=j makes the owner of column j never set its flag,
  // so every CTA's bounded wait for step j runs out (IE_WAIT_NS), the kernel records a
  // timeout and returns, and ie_create reports IE_ERR_TIMEOUT. Nothing faults or hangs.
  int64_t skip_publish = -1;
  if (const char* e = getenv("IE_TEST_SKIP_PUBLISH")) skip_publish = atoll(e);
  void* args[] = {&n, &kl, &ldab, &n_pad, &AB, &piv, &dinv, &ring, &ring_tp, &ring_flag, &R,
                  &status, &P, &nown_max, &skip_publish};
  ie_count_launch();
  return cudaLaunchCooperativeKernel((void*)kfn, dim3(q * P), dim3(512), args, smem, s);
}

cudaError_t launch_band_lu(int q, int64_t n, int kl, int ldab, int64_t n_pad, cplx* AB,
                           int* piv, cplx* dinv, cplx* ring, int* ring_tp, unsigned* ring_flag,
                           int R, int* status, cudaStream_t s, int* ctas_per_pole) {
  return band_lu_t(q, n, kl, ldab, n_pad, AB, piv, dinv, ring, ring_tp, ring_flag, R, status, s,
                   ctas_per_pole);
}

cudaError_t launch_band_lu(int q, int64_t n, int kl, int ldab, int64_t n_pad, float2* AB,
                           int* piv, float2* dinv, float2* ring, int* ring_tp,
                           unsigned* ring_flag, int R, int* status, cudaStream_t s,
                           int* ctas_per_pole) {
  return band_lu_t(q, n, kl, ldab, n_pad, AB, piv, dinv, ring, ring_tp, ring_flag, R, status, s,
                   ctas_per_pole);
}

// ----------------------------------------------------------------------------------------------
__global__ void pole_sum_kernel(int q, int64_t n, const cplx* Xp, int64_t ldx, int64_t xstride,
                                cplx* GV, int64_t ldg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= n) return;
  cplx acc = cmk(0, 0);
  for (int p = 0; p < q; ++p) acc = cadd(acc, Xp[(int64_t)p * xstride + (int64_t)c * ldx + i]);
  GV[(int64_t)c * ldg + i] = acc;
}

void launch_pole_sum(int q, int64_t n, int k, const cplx* Xp, int64_t ldx, int64_t xstride,
                     cplx* GV, int64_t ldg, cudaStream_t s) {
  if (k <= 0) return;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)k);
  pole_sum_kernel<<<grid, 256, 0, s>>>(q, n, Xp, ldx, xstride, GV, ldg); ie_count_launch();
}

// GV[:, c] = sum_i w_i Xp[i][:, c]
__global__ void pole_wsum_kernel(int q, int64_t n, const cplx* Xp, int64_t ldx, int64_t xstride,
                                 const cplx* w, cplx* GV, int64_t ldg) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= n) return;
  cplx acc = cmk(0, 0);
  for (int p = 0; p < q; ++p) acc = cfma(w[p], Xp[(int64_t)p * xstride + (int64_t)c * ldx + i], acc);
  GV[(int64_t)c * ldg + i] = acc;
}

void launch_pole_wsum(int q, int64_t n, int k, const cplx* Xp, int64_t ldx, int64_t xstride,
                      const cplx* w, cplx* GV, int64_t ldg, cudaStream_t s) {
  if (k <= 0) return;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)k);
  pole_wsum_kernel<<<grid, 256, 0, s>>>(q, n, Xp, ldx, xstride, w, GV, ldg); ie_count_launch();
}

// ----------------------------------------------------------------------------------------------
// Split factor layout for the solves: L column j = its kl multipliers (padded to klp), U column
// j = U(j-kv..j-1, j) (kv = 2 kl entries), columns contiguous per pole so that a panel of 8
// columns is one bulk copy with 16-byte aligned start and length. complex128 (from the LU in
// LAPACK band storage) or complex64 rounded from it (mixed precision, with 1/u_jj).
__device__ __forceinline__ cplx ld_c(const cplx* p) { return *p; }
__device__ __forceinline__ cplx ld_c(const float2* p) {
  const float2 v = *p;
  return make_double2(v.x, v.y);
}

// Split copy of band factors (input AB in complex128 or complex64, output in OT): L column j =
// its kl multipliers (padded to klp), U column j = U(j-kv..j-1, j); diag (nullable) = U(j,j).
template <typename IT, typename OT>
__global__ void factors_split_kernel(int64_t n_pad, int kl, int ldab, int klp, const IT* AB,
                                     OT* L, OT* U, OT* diag) {
  const int pole = blockIdx.y;
  const int kv = 2 * kl;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int per = klp + kv + 1;
  if (idx >= n_pad * per) return;
  const int64_t j = idx / per;
  const int t = (int)(idx - j * per);
  const IT* col = AB + ((int64_t)pole * n_pad + j) * ldab;
  if (t < klp) {
    put_c(&L[((int64_t)pole * n_pad + j) * klp + t], (t < kl) ? ld_c(col + kv + 1 + t) : cmk(0, 0));
  } else if (t < klp + kv) {
    put_c(&U[((int64_t)pole * n_pad + j) * kv + (t - klp)], ld_c(col + t - klp));
  } else if (diag) {
    put_c(&diag[(int64_t)pole * n_pad + j], ld_c(col + kv));
  }
}

void launch_factors_split32(int q, int64_t n_pad, int kl, int ldab, int klp, const float2* AB,
                            float2* L32, float2* U32, float2* diag32, cudaStream_t s) {
  const int64_t tot = n_pad * (klp + 2 * kl + 1);
  dim3 grid((unsigned)((tot + 255) / 256), (unsigned)q);
  factors_split_kernel<float2, float2><<<grid, 256, 0, s>>>(n_pad, kl, ldab, klp, AB, L32, U32, diag32); ie_count_launch();
}

void launch_factors_split64(int q, int64_t n_pad, int kl, int ldab, const cplx* AB, cplx* L64,
                            cplx* U64, cudaStream_t s) {
  const int64_t tot = n_pad * (kl + 2 * kl + 1);
  dim3 grid((unsigned)((tot + 255) / 256), (unsigned)q);
  factors_split_kernel<cplx, cplx><<<grid, 256, 0, s>>>(n_pad, kl, ldab, kl, AB, L64, U64, (cplx*)nullptr); ie_count_launch();
}

// R32[i][:, c] = (complex64) (BV[:, c] - K_i X[i][:, c]), K_i = p_i B - A, for all poles i:
// the FP64 residual of the mixed-precision refinement.
__global__ void pole_residual_kernel(DiaDev P, const cplx* poles, const cplx* BV, int64_t ldb,
                                     const cplx* X, int64_t ldx, int64_t xstride, float2* R32,
                                     int64_t ldr, int64_t rstride) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y, pole = blockIdx.z;
  if (i >= P.n) return;
  const cplx p = poles[pole];
  const cplx* x = X + (int64_t)pole * xstride + (int64_t)c * ldx;
  cplx acc = BV[(int64_t)c * ldb + i];
  for (int d = 0; d < P.ndiag; ++d) {
    const int64_t j = i + P.off[d];
    if (j < 0 || j >= P.n) continue;
    const cplx kij = csub(cmul(p, P.B[(int64_t)d * P.n + i]), P.A[(int64_t)d * P.n + i]);
    acc = cfms(kij, x[j], acc);
  }
  R32[(int64_t)pole * rstride + (int64_t)c * ldr + i] = make_float2((float)acc.x, (float)acc.y);
}

void launch_pole_residual(const DiaDev& P, const cplx* d_poles, int q, int k, const cplx* BV,
                          int64_t ldb, const cplx* X, int64_t ldx, int64_t xstride, float2* R32,
                          int64_t ldr, int64_t rstride, cudaStream_t s) {
  if (k <= 0) return;
  dim3 grid((unsigned)((P.n + 255) / 256), (unsigned)k, (unsigned)q);
  pole_residual_kernel<<<grid, 256, 0, s>>>(P, d_poles, BV, ldb, X, ldx, xstride, R32, ldr, rstride); ie_count_launch();
}

// Iterative-refinement update of the mixed-precision path: X[i][:, c] += D[i][:, c] (the FP32
// correction K~_i^{-1} r, widened to FP64), and per (pole, column) the largest |.|_1 entry of
// the correction and of the updated X, as float bits in nrm[(i*k + c)*2 + {0, 1}] (atomicMax on
// non-negative floats; the caller zeroes nrm). Their ratio estimates the relative error that the
// correction removed.
__global__ void refine_add_kernel(int64_t n, int k, const float2* D, int64_t ldd, int64_t dstride,
                                  cplx* X, int64_t ldx, int64_t xstride, unsigned* nrm) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y, pole = blockIdx.z;
  float md = 0.0f, mx = 0.0f;
  if (i < n) {
    const float2 d = D[(int64_t)pole * dstride + (int64_t)c * ldd + i];
    cplx* xp = X + (int64_t)pole * xstride + (int64_t)c * ldx + i;
    const cplx x = make_double2(xp->x + (double)d.x, xp->y + (double)d.y);
    *xp = x;
    md = fabsf(d.x) + fabsf(d.y);
    mx = (float)cabs1(x);
  }
  for (int o = 16; o > 0; o >>= 1) {
    md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
    mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  __shared__ float smd[8], smx[8];
  if ((threadIdx.x & 31) == 0) { smd[threadIdx.x >> 5] = md; smx[threadIdx.x >> 5] = mx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { md = fmaxf(md, smd[w]); mx = fmaxf(mx, smx[w]); }
    unsigned* o = nrm + ((int64_t)pole * k + c) * 2;
    atomicMax(o, __float_as_uint(md));
    atomicMax(o + 1, __float_as_uint(mx));
  }
}

void launch_refine_add(int q, int64_t n, int k, const float2* D, int64_t ldd, int64_t dstride,
                       cplx* X, int64_t ldx, int64_t xstride, unsigned* nrm, cudaStream_t s) {
  if (k <= 0) return;
  dim3 grid((unsigned)((n + 255) / 256), (unsigned)k, (unsigned)q);
  refine_add_kernel<<<grid, 256, 0, s>>>(n, k, D, ldd, dstride, X, ldx, xstride, nrm); ie_count_launch();
}

__global__ void to_c64_kernel(int64_t n, const cplx* X, int64_t ldx, float2* Y, int64_t ldy) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i >= n) return;
  const cplx v = X[(int64_t)c * ldx + i];
  Y[(int64_t)c * ldy + i] = make_float2((float)v.x, (float)v.y);
}

void launch_to_c64(int64_t n, int k, const cplx* X, int64_t ldx, float2* Y, int64_t ldy,
                   cudaStream_t s) {
  if (k <= 0) return;
  to_c64_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)k), 256, 0, s>>>(n, X, ldx, Y, ldy); ie_count_launch();
}

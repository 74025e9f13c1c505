// Band kernels of the inner operator G (Sec. 3.2, Eq. linearsolve2):
//   assembly of K_i = p_i B - A (Alg. 1 line 3) into LAPACK band storage,
//   batched band LU with partial pivoting over all q poles in one cooperative launch,
//   forward (P, L) + backward (U) band solves on n x k blocks with the factor panels
//   staged into shared memory by bulk asynchronous copies (TMA, cp.async.bulk),
//   the DIA SpMV with A and B, and the weighted pole sum.
#include <cooperative_groups.h>
#include <cstdio>

#include <atomic>

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
__global__ void assemble_kernel(DiaDev P, const cplx* poles, int kl, int ldab, int64_t n_pad,
                                cplx* AB) {
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
  AB[(int64_t)pole * n_pad * ldab + idx] = v;
}

void launch_assemble(const DiaDev& P, const cplx* d_poles, int q, int kl, int ldab,
                     int64_t n_pad, cplx* AB, cudaStream_t s) {
  const int64_t tot = n_pad * ldab;
  dim3 grid((unsigned)((tot + 255) / 256), (unsigned)q);
  assemble_kernel<<<grid, 256, 0, s>>>(P, d_poles, kl, ldab, n_pad, AB); ie_count_launch();
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
// Grid = q poles x P CTAs; CTA b owns the columns l with l % P == b. All CTAs of a pole read
// the pivot column and compute the pivot and multipliers redundantly; the owner of column j
// writes its final entries (U(j,j), L, piv, 1/pivot) after the step's barrier, when no CTA
// reads column j any more. One bounded per-pole barrier per column.

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_volatile_i32(const int* p) {
  return *(const volatile int*)p;
}

__device__ bool pole_barrier(unsigned* cnt, unsigned* gen, unsigned nb, unsigned& my_gen,
                             int* status) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned g = my_gen;
    __threadfence();
    if (atomicAdd(cnt, 1u) == nb - 1) {
      atomicExch(cnt, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      const unsigned long long t0 = ie_globaltimer();
      unsigned it = 0;
      while (ld_acquire_u32(gen) == g) {
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
    __threadfence();
    my_gen = g + 1;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

__global__ void __launch_bounds__(256) band_lu_kernel(int64_t n, int kl, int ldab, int64_t n_pad,
                                                      cplx* AB, int* piv, cplx* dinv,
                                                      unsigned* bar, int* status, int P,
                                                      int nown_max) {
  const int pole = blockIdx.x / P, b = blockIdx.x % P;
  const int T = blockDim.x, tid = threadIdx.x;
  const int kv = 2 * kl;
  cplx* A = AB + (int64_t)pole * n_pad * ldab;
  int* pv_out = piv + (int64_t)pole * n_pad;
  cplx* di_out = dinv + (int64_t)pole * n_pad;
  extern __shared__ double2 lu_sm[];
  cplx* col = lu_sm;                 // kl+1
  cplx* mult = col + (kl + 1);       // kl+1
  cplx* urow = mult + (kl + 1);      // nown_max
  cplx* arow = urow + nown_max;      // nown_max
  __shared__ double red_v[32];
  __shared__ int red_i[32];
  __shared__ int s_tp;
  unsigned* cnt = bar + 2 * pole;
  unsigned* gen = bar + 2 * pole + 1;
  unsigned my_gen = 0;
  int64_t ju = 0;
  int prev_tp = 0, prev_nrows = -1;
  cplx prev_pv = cmk(0, 0), prev_rcp = cmk(0, 0);

  for (int64_t j = 0; j < n; ++j) {
    // (a) final entries of column j-1, written by its owner once nobody reads it
    if (j > 0 && ((j - 1) % P) == b) {
      cplx* cj = A + (j - 1) * ldab + kv;
      for (int t = tid; t <= prev_nrows; t += T) cj[t] = (t == 0) ? prev_pv : mult[t];
      if (tid == 0) {
        pv_out[j - 1] = (int)(j - 1 + prev_tp);
        di_out[j - 1] = prev_rcp;
      }
    }
    __syncthreads();
    // (b) pivot column rows j..j+nrows
    const int nrows = (int)((n - 1 - j) < (int64_t)kl ? (n - 1 - j) : (int64_t)kl);
    const cplx* cj = A + j * ldab + kv;
    double best = -1.0;
    int bi = 0;
    for (int t = tid; t <= nrows; t += T) {
      const cplx v = __ldcg(cj + t);
      col[t] = v;
      const double a = cabs1(v);
      if (a > best) { best = a; bi = t; }
    }
    // (c) argmax, first index on ties
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if ((tid & 31) == 0) { red_v[tid >> 5] = best; red_i[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
      double bb = red_v[0];
      int ii = red_i[0];
      for (int w = 1; w < (T + 31) / 32; ++w)
        if (red_v[w] > bb || (red_v[w] == bb && red_i[w] < ii)) { bb = red_v[w]; ii = red_i[w]; }
      s_tp = ii;
    }
    __syncthreads();
    const int tp = s_tp;
    const cplx pv = col[tp];
    { const int64_t cand = (j + kl + tp < n - 1) ? (j + kl + tp) : (n - 1); if (cand > ju) ju = cand; }
    const bool zero = (pv.x == 0.0 && pv.y == 0.0);
    if (zero && b == 0 && tid == 0) atomicMax(status + ST_SINGULAR, 1);
    const cplx rcp = zero ? cmk(0, 0) : crcp(pv);
    for (int t = 1 + tid; t <= nrows; t += T)
      mult[t] = zero ? cmk(0, 0) : cmul((t == tp) ? col[0] : col[t], rcp);
    // (d) swap + rank-1 update of the owned columns l in (j, ju], l % P == b
    const int64_t jn = j + 1;
    const int64_t l0 = jn + (((int64_t)b - jn % P) % P + P) % P;
    const int nown = (!zero && l0 <= ju) ? (int)((ju - l0) / P + 1) : 0;
    for (int idx = tid; idx < nown; idx += T) {
      const int64_t l = l0 + (int64_t)idx * P;
      const cplx* cl = A + l * ldab + kv - (l - j);   // row j of column l
      urow[idx] = __ldcg(cl + tp);
      arow[idx] = __ldcg(cl);
    }
    __syncthreads();
    if (nown > 0 && nrows > 0) {
      const int tot = nrows * nown;
      for (int it = tid; it < tot; it += T) {
        const int idx = it / nrows;
        const int t = 1 + (it - idx * nrows);
        const int64_t l = l0 + (int64_t)idx * P;
        cplx* cl = A + l * ldab + kv - (l - j);
        cplx v = (t == tp) ? arow[idx] : __ldcg(cl + t);
        cl[t] = cfms(mult[t], urow[idx], v);
      }
    }
    for (int idx = tid; idx < nown; idx += T) {
      const int64_t l = l0 + (int64_t)idx * P;
      A[l * ldab + kv - (l - j)] = urow[idx];
    }
    prev_tp = tp;
    prev_nrows = nrows;
    prev_pv = pv;
    prev_rcp = rcp;
    if (!pole_barrier(cnt, gen, (unsigned)P, my_gen, status)) return;
  }
  if (n > 0 && ((n - 1) % P) == b) {
    cplx* cj = A + (n - 1) * ldab + kv;
    for (int t = tid; t <= prev_nrows; t += T) cj[t] = (t == 0) ? prev_pv : mult[t];
    if (tid == 0) {
      pv_out[n - 1] = (int)(n - 1 + prev_tp);
      di_out[n - 1] = prev_rcp;
    }
  }
}

cudaError_t launch_band_lu(int q, int64_t n, int kl, int ldab, int64_t n_pad, cplx* AB,
                           int* piv, cplx* dinv, unsigned* bar, int* status, cudaStream_t s,
                           int* ctas_per_pole) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int kv = 2 * kl;
  int P = sms / q;
  if (P < 1) P = 1;
  if (P > kv) P = kv;
  if (P < 1) P = 1;
  int nown_max = (kv + P - 1) / P + 1;
  size_t smem = (size_t)(2 * (kl + 1) + 2 * nown_max) * sizeof(cplx);
  if (smem > 48 * 1024)
    cudaFuncSetAttribute(band_lu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, band_lu_kernel, 256, smem);
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  while ((int64_t)P * q > (int64_t)per_sm * sms && P > 1) {
    --P;
    nown_max = (kv + P - 1) / P + 1;
  }
  smem = (size_t)(2 * (kl + 1) + 2 * nown_max) * sizeof(cplx);
  if (ctas_per_pole) *ctas_per_pole = P;
  cudaMemsetAsync(bar, 0, sizeof(unsigned) * 2 * q, s);
  void* args[] = {&n, &kl, &ldab, &n_pad, &AB, &piv, &dinv, &bar, &status, &P, &nown_max};
  ie_count_launch();
  return cudaLaunchCooperativeKernel((void*)band_lu_kernel, dim3(q * P), dim3(256), args, smem, s);
}

// ----------------------------------------------------------------------------------------------
// Band solves. One CTA per (pole, group of NC right-hand-side columns); the row recurrence is
// sequential in n, so parallelism comes from poles x column groups and from the band width
// inside each step. The active window of the recurrence lives in registers, one row slot per
// thread (slot = row mod S): forward S = kl+1 rows j..j+kl, backward S = kv+1 rows j-kv..j.
// Per step: the pivot/diagonal values are broadcast through a double-buffered shared cell,
// every slot does NC complex FMAs with one factor entry, one __syncthreads.
// Factor columns are staged NB at a time into an NSTAGE-deep shared ring by cp.async.bulk
// (L parts for the forward sweep, U parts for the backward sweep), completion tracked by
// mbarriers; all waits are bounded.

namespace {
constexpr int SOLVE_NB = 4;   // factor columns per staged panel (multiple of 4: 16-byte int copies)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: false after IE_WAIT_NS
__device__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = ie_globaltimer();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_try_wait(bar, parity)) return true;
    if (ie_globaltimer() - t0 > IE_WAIT_NS) return false;
  }
}
}  // namespace

struct SolveArgs {
  int64_t n, n_pad, ldab, ldr, ldx, xstride;
  int kl, kv, k, nstage;
  const cplx* AB;
  const int* piv;
  const cplx* dinv;
  const cplx* weights;
  const cplx* RHS;
  cplx* X;
  int* status;
};

template <int NC, int SPT>
__global__ void __launch_bounds__(640, 1) band_solve_kernel(SolveArgs a) {
  const int pole = blockIdx.y;
  const int c0 = blockIdx.x * NC;
  const int ncol = min(NC, a.k - c0);
  const int T = blockDim.x, tid = threadIdx.x;
  const int kl = a.kl, kv = a.kv;
  const int64_t n = a.n;
  const cplx* ABp = a.AB + (int64_t)pole * a.n_pad * a.ldab;
  const int* pivp = a.piv + (int64_t)pole * a.n_pad;
  const cplx* dinvp = a.dinv + (int64_t)pole * a.n_pad;
  cplx* Xo = a.X + (int64_t)pole * a.xstride;
  const cplx* R = a.RHS;
  const cplx w = a.weights[pole];

  extern __shared__ __align__(128) unsigned char sm_raw[];
  uint64_t* mbar = (uint64_t*)sm_raw;                      // nstage mbarriers
  cplx* bc = (cplx*)(sm_raw + 128);                        // [2][2][NC] broadcast cells
  unsigned char* stage0 = sm_raw + 128 + 4 * NC * sizeof(cplx) + 128;
  stage0 = (unsigned char*)(((uintptr_t)stage0 + 127) & ~(uintptr_t)127);
  const int NB = SOLVE_NB;
  const size_t fwd_cols_bytes = (size_t)NB * kl * sizeof(cplx);
  const size_t bwd_cols_bytes = (size_t)NB * kv * sizeof(cplx);
  const size_t stage_bytes = ((bwd_cols_bytes + NB * sizeof(cplx)) + 127) & ~(size_t)127;
  __shared__ int s_fail;

  if (tid == 0) {
    s_fail = 0;
    for (int i = 0; i < a.nstage; ++i) mbar_init(smem_u32(&mbar[i]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const int64_t npanel = a.n_pad / NB;
  // ------------------------------- forward: P L y = rhs -------------------------------------
  auto issue_fwd = [&](int64_t P, int st) {
    unsigned char* dst = stage0 + (size_t)st * stage_bytes;
    const uint32_t bar = smem_u32(&mbar[st]);
    const uint32_t bytes = (uint32_t)(fwd_cols_bytes + NB * sizeof(int));
    mbar_expect_tx(bar, bytes);
    for (int jj = 0; jj < NB; ++jj) {
      const int64_t col = P * NB + jj;
      bulk_g2s(smem_u32(dst + (size_t)jj * kl * sizeof(cplx)), ABp + col * a.ldab + kv + 1,
               (uint32_t)(kl * sizeof(cplx)), bar);
    }
    bulk_g2s(smem_u32(dst + fwd_cols_bytes), pivp + P * NB, (uint32_t)(NB * sizeof(int)), bar);
  };
  const int S = kl + 1;
  cplx v[SPT][NC], nxt[SPT][NC];
  int off[SPT];
  if (tid == 0)
    for (int st = 0; st < a.nstage && st < npanel; ++st) issue_fwd(st, st);
  {
    const int p0 = __ldg(pivp);
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      const int s = tid + u * T;
      off[u] = s;
      const int64_t r = s;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        v[u][c] = (s < S && r < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + r] : cmk(0, 0);
        nxt[u][c] = (s < S && r + S < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + r + S]
                                                     : cmk(0, 0);
      }
      if (s < S) {
        if (r == p0)
#pragma unroll
          for (int c = 0; c < NC; ++c) bc[0 * 2 * NC + 0 * NC + c] = v[u][c];
        if (r == 0)
#pragma unroll
          for (int c = 0; c < NC; ++c) bc[0 * 2 * NC + 1 * NC + c] = v[u][c];
      }
    }
  }
  __syncthreads();
  bool failed = false;
  for (int64_t P = 0; P < npanel && !failed; ++P) {
    const int st = (int)(P % a.nstage);
    if (!mbar_wait_bounded(smem_u32(&mbar[st]), (uint32_t)((P / a.nstage) & 1))) s_fail = 1;
    __syncthreads();
    if (s_fail) { failed = true; break; }
    const cplx* Lst = (const cplx*)(stage0 + (size_t)st * stage_bytes);
    const int* pst = (const int*)(stage0 + (size_t)st * stage_bytes + fwd_cols_bytes);
    for (int jj = 0; jj < NB; ++jj) {
      const int64_t j = P * NB + jj;
      if (j >= n) break;
      const int par = (int)(j & 1);
      cplx x[NC], xj[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        x[c] = bc[par * 2 * NC + c];
        xj[c] = bc[par * 2 * NC + NC + c];
      }
      const int64_t jp = pst[jj];
      const int64_t jp1 = (j + 1 < n) ? ((jj + 1 < NB) ? pst[jj + 1] : __ldg(pivp + j + 1)) : -1;
      const cplx* Lc = Lst + (size_t)jj * kl;
#pragma unroll
      for (int u = 0; u < SPT; ++u) {
        const int s = tid + u * T;
        if (s >= S) continue;
        const int o = off[u];
        int64_t rnew;
        if (o == 0) {
          // row j leaves: y_j = x; slot refilled with row j + S
#pragma unroll
          for (int c = 0; c < NC; ++c)
            if (c < ncol) Xo[(int64_t)(c0 + c) * a.ldx + j] = x[c];
          rnew = j + S;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            v[u][c] = nxt[u][c];
            nxt[u][c] = (rnew + S < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + rnew + S]
                                                   : cmk(0, 0);
          }
          off[u] = S - 1;
        } else {
          const int64_t r = j + o;
          const cplx l = Lc[o - 1];
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            cplx t = (r == jp) ? xj[c] : v[u][c];
            v[u][c] = cfms(l, x[c], t);
          }
          off[u] = o - 1;
          rnew = r;
        }
        const int npar = par ^ 1;
        if (rnew == jp1)
#pragma unroll
          for (int c = 0; c < NC; ++c) bc[npar * 2 * NC + c] = v[u][c];
        if (rnew == j + 1)
#pragma unroll
          for (int c = 0; c < NC; ++c) bc[npar * 2 * NC + NC + c] = v[u][c];
      }
      __syncthreads();
    }
    if (tid == 0 && P + a.nstage < npanel) issue_fwd(P + a.nstage, st);
  }
  if (failed) {
    if (tid == 0) atomicExch(a.status + ST_TIMEOUT, 1);
    // wait (bounded) for the copies that may still be in flight, then leave
    for (int st = 0; st < a.nstage; ++st)
      for (int ph = 0; ph < 2; ++ph) mbar_wait_bounded(smem_u32(&mbar[st]), (uint32_t)ph);
    return;
  }
  __syncthreads();
  // re-initialise the barriers for the backward sweep (every forward stage has completed)
  if (tid == 0) {
    for (int i = 0; i < a.nstage; ++i) {
      asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&mbar[i])) : "memory");
      mbar_init(smem_u32(&mbar[i]), 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  // ------------------------------- backward: U x = y ----------------------------------------
  // panel B covers columns [n_pad - (B+1) NB, n_pad - B NB)
  auto issue_bwd = [&](int64_t Bp, int st) {
    unsigned char* dst = stage0 + (size_t)st * stage_bytes;
    const uint32_t bar = smem_u32(&mbar[st]);
    const int64_t cb0 = a.n_pad - (Bp + 1) * NB;
    const uint32_t bytes = (uint32_t)(bwd_cols_bytes + NB * sizeof(cplx));
    mbar_expect_tx(bar, bytes);
    for (int jj = 0; jj < NB; ++jj)
      bulk_g2s(smem_u32(dst + (size_t)jj * kv * sizeof(cplx)), ABp + (cb0 + jj) * a.ldab,
               (uint32_t)(kv * sizeof(cplx)), bar);
    bulk_g2s(smem_u32(dst + bwd_cols_bytes), dinvp + cb0, (uint32_t)(NB * sizeof(cplx)), bar);
  };
  const int Sb = kv + 1;
  if (tid == 0)
    for (int st = 0; st < a.nstage && st < npanel; ++st) issue_bwd(st, st);
  {
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      const int s = tid + u * T;
      int o = (int)(((n - 1 - s) % Sb + Sb) % Sb);
      off[u] = o;
      const int64_t r = n - 1 - o;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        v[u][c] = (s < Sb && r >= 0 && c < ncol) ? Xo[(int64_t)(c0 + c) * a.ldx + r] : cmk(0, 0);
        nxt[u][c] = (s < Sb && r - Sb >= 0 && c < ncol) ? Xo[(int64_t)(c0 + c) * a.ldx + r - Sb]
                                                        : cmk(0, 0);
      }
      if (s < Sb && r == n - 1) {
        const int par = (int)((n - 1) & 1);
#pragma unroll
        for (int c = 0; c < NC; ++c) bc[par * 2 * NC + c] = v[u][c];
      }
    }
  }
  __syncthreads();
  for (int64_t Bp = 0; Bp < npanel && !failed; ++Bp) {
    const int st = (int)(Bp % a.nstage);
    if (!mbar_wait_bounded(smem_u32(&mbar[st]), (uint32_t)((Bp / a.nstage) & 1))) s_fail = 1;
    __syncthreads();
    if (s_fail) { failed = true; break; }
    const cplx* Ust = (const cplx*)(stage0 + (size_t)st * stage_bytes);
    const cplx* dst_ = (const cplx*)(stage0 + (size_t)st * stage_bytes + bwd_cols_bytes);
    const int64_t cb0 = a.n_pad - (Bp + 1) * NB;
    for (int jj = NB - 1; jj >= 0; --jj) {
      const int64_t j = cb0 + jj;
      if (j >= n) continue;
      const int par = (int)(j & 1);
      const cplx dj = dst_[jj];
      cplx xj[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) xj[c] = cmul(bc[par * 2 * NC + c], dj);
      const cplx* Uc = Ust + (size_t)jj * kv;
#pragma unroll
      for (int u = 0; u < SPT; ++u) {
        const int s = tid + u * T;
        if (s >= Sb) continue;
        const int o = off[u];
        int64_t rnew;
        if (o == 0) {
#pragma unroll
          for (int c = 0; c < NC; ++c)
            if (c < ncol) Xo[(int64_t)(c0 + c) * a.ldx + j] = cmul(w, xj[c]);
          rnew = j - Sb;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            v[u][c] = nxt[u][c];
            nxt[u][c] = (rnew - Sb >= 0 && c < ncol) ? Xo[(int64_t)(c0 + c) * a.ldx + rnew - Sb]
                                                     : cmk(0, 0);
          }
          off[u] = kv;
        } else {
          const cplx uu = Uc[kv - o];
#pragma unroll
          for (int c = 0; c < NC; ++c) v[u][c] = cfms(uu, xj[c], v[u][c]);
          off[u] = o - 1;
          rnew = j - o;
        }
        if (rnew == j - 1) {
          const int npar = par ^ 1;
#pragma unroll
          for (int c = 0; c < NC; ++c) bc[npar * 2 * NC + c] = v[u][c];
        }
      }
      __syncthreads();
    }
    if (tid == 0 && Bp + a.nstage < npanel) issue_bwd(Bp + a.nstage, st);
  }
  if (failed) {
    if (tid == 0) atomicExch(a.status + ST_TIMEOUT, 1);
    for (int st = 0; st < a.nstage; ++st)
      for (int ph = 0; ph < 2; ++ph) mbar_wait_bounded(smem_u32(&mbar[st]), (uint32_t)ph);
  }
}

template <int NC, int SPT>
static cudaError_t launch_solve_t(const SolveArgs& a, int q, int threads, size_t smem,
                                  cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(band_solve_kernel<NC, SPT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)((a.k + NC - 1) / NC), (unsigned)q);
  band_solve_kernel<NC, SPT><<<grid, threads, smem, s>>>(a); ie_count_launch();
  return cudaGetLastError();
}

cudaError_t launch_band_solve(int q, int64_t n, int kl, int ldab, int64_t n_pad, const cplx* AB,
                              const int* piv, const cplx* dinv, const cplx* d_weights,
                              const cplx* RHS, int64_t ldr, int k, cplx* Xp, int64_t ldx,
                              int64_t xstride, int* status, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  SolveArgs a;
  a.n = n; a.n_pad = n_pad; a.ldab = ldab; a.ldr = ldr; a.ldx = ldx; a.xstride = xstride;
  a.kl = kl; a.kv = 2 * kl; a.k = k;
  a.AB = AB; a.piv = piv; a.dinv = dinv; a.weights = d_weights; a.RHS = RHS; a.X = Xp;
  a.status = status;
  const int slots = a.kv + 1;
  const int spt = slots > 640 ? 2 : 1;
  if (slots > 1280) return cudaErrorInvalidValue;   // half bandwidth up to 639
  int threads = ((slots + spt - 1) / spt + 31) / 32 * 32;
  const size_t stage_bytes =
      (((size_t)SOLVE_NB * a.kv * sizeof(cplx) + SOLVE_NB * sizeof(cplx)) + 127) & ~(size_t)127;
  const size_t fixed = 128 + 4 * 4 * sizeof(cplx) + 128 + 128;
  const size_t budget = 200 * 1024;
  int nstage = (int)((budget - fixed) / stage_bytes);
  if (nstage > 6) nstage = 6;
  if (nstage < 2) return cudaErrorInvalidValue;
  a.nstage = nstage;
  const size_t smem = fixed + (size_t)nstage * stage_bytes;
  // columns per CTA: the smallest NC that keeps q * ceil(k/NC) CTAs within one wave
  int NC = 4;
  for (int c = 1; c <= 4; ++c)
    if ((int64_t)q * ((k + c - 1) / c) <= sms) { NC = c; break; }
  if (spt == 1) {
    switch (NC) {
      case 1: return launch_solve_t<1, 1>(a, q, threads, smem, s);
      case 2: return launch_solve_t<2, 1>(a, q, threads, smem, s);
      case 3: return launch_solve_t<3, 1>(a, q, threads, smem, s);
      default: return launch_solve_t<4, 1>(a, q, threads, smem, s);
    }
  } else {
    switch (NC) {
      case 1: return launch_solve_t<1, 2>(a, q, threads, smem, s);
      case 2: return launch_solve_t<2, 2>(a, q, threads, smem, s);
      default: return launch_solve_t<4, 2>(a, q, threads, smem, s);
    }
  }
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

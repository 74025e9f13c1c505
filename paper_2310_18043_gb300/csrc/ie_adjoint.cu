// Adjoint pencil and eigenvalue sensitivities (an extension of the paper's method: it
// computes right eigenpairs only).
//
// Left eigenvectors of (A, B) are right eigenvectors of (A^H, B^H) on the conjugate disk.
// The inner operator of that pencil, G_adj(V) = sum_i conj(w_i) K_i^{-H} B^H V, reuses the
// band LU of each K_i = p_i B - A (K_i = P_i^T L_i U_i in LAPACK zgbtrf form):
//   K_i^{-H} z = P_i^T L_i^{-H} U_i^{-H} z,
// solved like LAPACK zgbtrs with trans = 'C': first U^H w = z (lower triangular, band
// 2 kl, non-unit), then for j = n-1 .. 0: w_j -= sum_{r=j+1}^{j+kl} conj(L(r,j)) w_r,
// followed by the swap of w_j and w_{piv(j)}.
//
// Kernel design (one CTA per (pole, group of NC right-hand sides), all q poles and k
// columns in one launch, factor panels of 8 staged by cp.async.bulk with bounded waits):
//  phase 1, U^H forward, ascending blocks of 8 rows: the window of kv + 8 rows lives in
//    registers (one row slot per thread and column); the 8 head rows are solved with the
//    precomputed inverse of U's 8x8 diagonal block (conjugate-transposed), then every other
//    slot subtracts the block's 8 contributions at once. It reads U by rows, so U is kept
//    a second time in row-major band form (row j: U(j, j+1..j+kv), built once).
//  phase 2, L^H backward with the pivots, descending blocks: the window of kl + 8 rows is in
//    shared memory. A block's 8 steps touch, besides reading, only the set H of its head
//    rows and pivot rows (16 members, the same set as the forward transform). Every other
//    window row enters only through the 8 dot products d_jj = sum conj(L(r, j)) w_r over
//    non-member rows, computed by thread groups with a shuffle reduction. The block is then
//    H <- M1 H + M2 d with a precomputed 16x24 matrix M = [M1 M2] per panel.
#include <algorithm>

#include "ie_internal.cuh"
#include "ie_bulk.cuh"

using namespace iebulk;

namespace {
constexpr int NB = 8;    // rows per block = factor columns per staged panel
constexpr int MW = 24;   // columns of a panel's phase-2 transform: 16 members + 8 dot inputs

__device__ __forceinline__ double2 shfl_xor_c(double2 v, int off, int width) {
  return make_double2(__shfl_xor_sync(0xffffffffu, v.x, off, width),
                      __shfl_xor_sync(0xffffffffu, v.y, off, width));
}
__device__ __forceinline__ float2 shfl_xor_c(float2 v, int off, int width) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, off, width),
                     __shfl_xor_sync(0xffffffffu, v.y, off, width));
}
__device__ __forceinline__ double2 cadd_t(double2 a, double2 b) { return cadd(a, b); }
__device__ __forceinline__ float2 cadd_t(float2 a, float2 b) {
  return make_float2(a.x + b.x, a.y + b.y);
}
__device__ __forceinline__ void put_c(cplx* p, cplx v) { *p = v; }
__device__ __forceinline__ void put_c(float2* p, cplx v) {
  *p = make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ cplx ld_c(const cplx* p) { return *p; }
__device__ __forceinline__ cplx ld_c(const float2* p) {
  const float2 v = *p;
  return make_double2(v.x, v.y);
}
}  // namespace

// ----------------------------------------------------------------------------------------------
// (A^H, B^H) in DIA form with the same diagonal order: offset -o, entry i = conj(M[i - o, i]).
__global__ void dia_adjoint_kernel(DiaDev P, cplx* AH, cplx* BH) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int d = blockIdx.y;
  if (i >= P.n) return;
  const int64_t src = i - P.off[d];
  const bool ok = src >= 0 && src < P.n;
  AH[(int64_t)d * P.n + i] = ok ? cconj(P.A[(int64_t)d * P.n + src]) : cmk(0, 0);
  BH[(int64_t)d * P.n + i] = ok ? cconj(P.B[(int64_t)d * P.n + src]) : cmk(0, 0);
}

void launch_dia_adjoint(const DiaDev& P, cplx* AH, cplx* BH, DiaDev* PH, cudaStream_t s) {
  dim3 grid((unsigned)((P.n + 255) / 256), (unsigned)P.ndiag);
  dia_adjoint_kernel<<<grid, 256, 0, s>>>(P, AH, BH); ie_count_launch();
  *PH = P;
  for (int d = 0; d < P.ndiag; ++d) PH->off[d] = -P.off[d];
  PH->A = AH;
  PH->B = BH;
}

// U by rows: Ut[pole][j][d-1] = U(j, j+d), d = 1..kv (zero past the matrix).
template <typename AT, typename OT>
__global__ void u_rows_kernel(int64_t n, int64_t n_pad, int kl, int ldab, const AT* AB, OT* Ut) {
  const int pole = blockIdx.y;
  const int kv = 2 * kl;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n_pad * kv) return;
  const int64_t j = idx / kv;
  const int d = (int)(idx - j * kv) + 1;
  cplx v = cmk(0, 0);
  if (j < n && j + d < n) v = ld_c(AB + ((int64_t)pole * n_pad + j + d) * ldab + kv - d);
  put_c(&Ut[((int64_t)pole * n_pad + j) * kv + d - 1], v);
}

void launch_u_rows(int q, int64_t n, int64_t n_pad, int kl, int ldab, const cplx* AB, cplx* Ut64,
                   float2* Ut32, cudaStream_t s) {
  const int64_t tot = n_pad * 2 * kl;
  dim3 grid((unsigned)((tot + 255) / 256), (unsigned)q);
  if (Ut64) { u_rows_kernel<cplx, cplx><<<grid, 256, 0, s>>>(n, n_pad, kl, ldab, AB, Ut64); ie_count_launch(); }
  if (Ut32) { u_rows_kernel<cplx, float2><<<grid, 256, 0, s>>>(n, n_pad, kl, ldab, AB, Ut32); ie_count_launch(); }
}

void launch_u_rows(int q, int64_t n, int64_t n_pad, int kl, int ldab, const float2* AB,
                   float2* Ut32, cudaStream_t s) {
  const int64_t tot = n_pad * 2 * kl;
  dim3 grid((unsigned)((tot + 255) / 256), (unsigned)q);
  u_rows_kernel<float2, float2><<<grid, 256, 0, s>>>(n, n_pad, kl, ldab, AB, Ut32); ie_count_launch();
}

// Phase-2 transform of each (panel, pole), one warp: lanes 0..15 carry the values of the
// members H (Hb, the forward transform's member rows). Input column m < 16 is member m's
// unit vector, column 16 + jj the dot input d_jj; the panel's steps are run in reverse
// (jj = nvalid-1 .. 0): member j0+jj subtracts sum conj(L(r, j)) v_r over the members r in
// (j, j+kl] and d_jj, then swaps with its pivot row. M[l][m] = final value of member l.
template <typename AT>
__global__ void adj_transform_kernel(int64_t n, int64_t n_pad, int kl, int ldab, const AT* AB,
                                     const int* piv, const int* Hb, cplx* Mout, float2* M32) {
  const int P = blockIdx.x, pole = blockIdx.y, lane = threadIdx.x;
  const int kv = 2 * kl;
  const int64_t npan = n_pad / NB;
  const int64_t j0 = (int64_t)P * NB;
  const int nvalid = (int)((n - j0) < NB ? (n - j0) : NB);
  const AT* A = AB + (int64_t)pole * n_pad * ldab;
  const int* pv = piv + (int64_t)pole * n_pad;
  const int64_t base = (int64_t)pole * npan + P;
  const int* H = Hb + base * 16;
  const int64_t myrow = (lane < 16) ? (int64_t)H[lane] : -1;
  int pm[NB];
#pragma unroll
  for (int jj = 0; jj < NB; ++jj) {
    pm[jj] = -1;
    if (jj < nvalid)
      for (int l = 0; l < 16; ++l)
        if (H[l] == pv[j0 + jj]) { pm[jj] = l; break; }
  }
  for (int m = 0; m < MW; ++m) {
    const bool present = (m < 16) ? (H[m] >= 0) : (m - 16 < nvalid);
    cplx val = make_double2((lane == m && m < 16 && present) ? 1.0 : 0.0, 0.0);
    if (present) {
      for (int jj = nvalid - 1; jj >= 0; --jj) {
        const int64_t j = j0 + jj;
        cplx t = make_double2(0, 0);
        if (myrow > j && myrow <= j + kl && myrow < n)
          t = cmul(cconj(ld_c(A + j * ldab + kv + (myrow - j))), val);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
          t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
        }
        if (lane == jj) {
          val = csub(val, t);
          if (m == 16 + jj) val.x -= 1.0;
        }
        const int b = pm[jj];
        const double vjx = __shfl_sync(0xffffffffu, val.x, jj), vjy = __shfl_sync(0xffffffffu, val.y, jj);
        const int bb = b < 0 ? jj : b;
        const double vbx = __shfl_sync(0xffffffffu, val.x, bb), vby = __shfl_sync(0xffffffffu, val.y, bb);
        if (b >= 0 && b != jj) {
          if (lane == jj) val = make_double2(vbx, vby);
          else if (lane == b) val = make_double2(vjx, vjy);
        }
      }
    }
    if (lane < 16) {
      const cplx o = (myrow >= 0 && present) ? val : make_double2(0, 0);
      if (Mout) Mout[base * (16 * MW) + lane * MW + m] = o;
      if (M32) M32[base * (16 * MW) + lane * MW + m] = make_float2((float)o.x, (float)o.y);
    }
  }
}

void launch_adj_transforms(int q, int64_t n, int64_t n_pad, int kl, int ldab, const cplx* AB,
                           const int* piv, const int* Hb, cplx* M64, float2* M32, cudaStream_t s) {
  dim3 grid((unsigned)(n_pad / NB), (unsigned)q);
  adj_transform_kernel<cplx><<<grid, 32, 0, s>>>(n, n_pad, kl, ldab, AB, piv, Hb, M64, M32); ie_count_launch();
}

void launch_adj_transforms(int q, int64_t n, int64_t n_pad, int kl, int ldab, const float2* AB,
                           const int* piv, const int* Hb, float2* M32, cudaStream_t s) {
  dim3 grid((unsigned)(n_pad / NB), (unsigned)q);
  adj_transform_kernel<float2><<<grid, 32, 0, s>>>(n, n_pad, kl, ldab, AB, piv, Hb, nullptr, M32); ie_count_launch();
}

// ----------------------------------------------------------------------------------------------
template <typename CT>
struct AdjArgsT {
  int64_t n, n_pad;
  int kl, kv, klp, kvp, k, nstage, mode;
  const CT* L;        // split L columns: column j's kl multipliers at L + pole*lstride + j*ldl
  int64_t ldl, lstride;
  const CT* Ut;       // U rows: row j's U(j, j+1..j+kv) at Ut + pole*ustride + j*ldu (ldu = kvp)
  int64_t ldu, ustride;
  const CT* Ub;       // [pole][panel][8][8] inverse of U's diagonal block, (i, b) at i*8 + b
  const CT* Mb;       // [pole][panel][16][24] phase-2 transforms
  const int* Hb;      // [pole][panel][16] member rows
  const cplx* weights;
  const CT* RHS;      // column c at RHS + pole*rstride + c*ldr
  int64_t ldr, rstride;
  CT* Y;              // phase-1 result (and, mode 0, the output), column c at Y + pole*ystride + c*ldy
  int64_t ldy, ystride;
  cplx* X;            // output for mode 1 (X = x); mode 3 writes x in place into Y
  int64_t ldx, xstride;
  int* status;
};

template <typename CT, int NC, int SPT, int REGS>
__global__ void __maxnreg__(REGS) band_solve_adj_kernel(AdjArgsT<CT> a) {
  const int pole = blockIdx.y;
  const int c0 = blockIdx.x * NC;
  const int ncol = min(NC, a.k - c0);
  const int T = blockDim.x, tid = threadIdx.x;
  const int kl = a.kl, kv = a.kv, klp = a.klp, kvp = a.kvp;
  const int64_t n = a.n;
  const int64_t npanel = a.n_pad / NB;
  const CT* Lp = a.L + (int64_t)pole * a.lstride;
  const CT* Utp = a.Ut + (int64_t)pole * a.ustride;
  const CT* Uip = a.Ub + (int64_t)pole * npanel * 64;
  const CT* Mp = a.Mb + (int64_t)pole * npanel * (16 * MW);
  const int* Hp = a.Hb + (int64_t)pole * npanel * 16;
  const CT* R = a.RHS + (int64_t)pole * a.rstride;
  CT* Yo = a.Y + (int64_t)pole * a.ystride;
  cplx* Xo = a.X + (int64_t)pole * a.xstride;
  const cplx w = a.weights[pole];
  const CT zero{};
  const int S2 = kl + NB;

  extern __shared__ __align__(128) unsigned char sm_raw[];
  uint64_t* mbar = (uint64_t*)sm_raw;                          // nstage mbarriers
  CT* hd = (CT*)(sm_raw + 128);                                // [NB][NC] head values
  CT* xs = hd + NB * NC;                                       // [NB][NC] solved head
  CT* hv = xs + NB * NC;                                       // [16][NC] members
  CT* dv = hv + 16 * NC;                                       // [NB][NC] dot inputs
  CT* part = dv + NB * NC;                                     // [NPART][NB][NC] partials
  CT* win = part + NPART * NB * NC;                            // [S2][NC] phase-2 window
  unsigned char* mflag = (unsigned char*)(win + (size_t)S2 * NC);   // [S2] member marks
  unsigned char* stage0 = (unsigned char*)(((uintptr_t)(mflag + S2) + 127) & ~(uintptr_t)127);
  const size_t p1_cols = (size_t)NB * kvp * sizeof(CT);
  const size_t p1_bytes = p1_cols + 64 * sizeof(CT);
  const size_t p2_cols = (size_t)NB * klp * sizeof(CT);
  const size_t p2_bytes = p2_cols + 16 * MW * sizeof(CT) + 16 * sizeof(int);
  const size_t stage_bytes = ((p1_bytes > p2_bytes ? p1_bytes : p2_bytes) + 127) & ~(size_t)127;
  __shared__ int s_fail;
  {
    // the staged ring must lie inside the dynamic allocation; refuse to run otherwise
    unsigned dsz;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsz));
    if ((size_t)(stage0 - sm_raw) + (size_t)a.nstage * stage_bytes > (size_t)dsz) {
      if (tid == 0) atomicExch(a.status + ST_TIMEOUT, 1);
      return;
    }
  }
  auto out = [&](int64_t r, int c, CT xv) {
    if constexpr (sizeof(CT) == sizeof(cplx)) {
      if (a.mode == 0) {
        Yo[(int64_t)(c0 + c) * a.ldy + r] = cmul(w, to_d(xv));
        return;
      }
    }
    if (a.mode == 1) {
      Xo[(int64_t)(c0 + c) * a.ldx + r] = to_d(xv);
    } else if (a.mode == 3) {
      Yo[(int64_t)(c0 + c) * a.ldy + r] = xv;   // in place, as mode 0: row r is no longer read
    }
  };

  if (tid == 0) {
    s_fail = 0;
    for (int i = 0; i < a.nstage; ++i) mbar_init(smem_u32(&mbar[i]), 1);
    mbar_fence_init();
  }
  for (int i = tid; i < S2; i += T) mflag[i] = 0;

  // ------------------------------- phase 1: U^H w = rhs ---------------------------------------
  // Block = panel P, head rows j0..j0+7 in hd (shared memory); the register window holds the
  // rows the panel updates, j0+8..j0+7+kv, Sf = max(kv, NB) slots (slot = (row - NB) mod Sf).
  // After the update the window's first NB rows become the next head and their slots take
  // the rows entering the window. Stage: U rows j0..j0+7 (contiguous) and the panel's
  // inverse diagonal block.
  auto issue1 = [&](int64_t P, int st) {
    unsigned char* dst = stage0 + (size_t)st * stage_bytes;
    const uint32_t bar = smem_u32(&mbar[st]);
    mbar_expect_tx(bar, (uint32_t)p1_bytes);
    bulk_g2s(smem_u32(dst), Utp + P * NB * a.ldu, (uint32_t)p1_cols, bar);
    bulk_g2s(smem_u32(dst + p1_cols), Uip + P * 64, (uint32_t)(64 * sizeof(CT)), bar);
  };
  const int Sf = kv > NB ? kv : NB;
  CT v[SPT][NC], nxt[SPT][NC];
  int64_t row[SPT];
  if (tid == T - 32)
    for (int st = 0; st < a.nstage && st < npanel; ++st) issue1(st, st);
  for (int e = tid; e < NB * NC; e += T) {
    const int t = e / NC, c = e - (e / NC) * NC;
    hd[e] = (t < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + t] : zero;
  }
#pragma unroll
  for (int u = 0; u < SPT; ++u) {
    const int s = tid + u * T;
    const int64_t r = NB + s;
    row[u] = r;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      v[u][c] = (s < Sf && r < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + r] : zero;
      nxt[u][c] = (s < Sf && r + Sf < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + r + Sf] : zero;
    }
  }
  __syncthreads();
  bool failed = false;
  // stage ring position and mbarrier phase as running 32-bit counters (no division per panel)
  int st = 0, stp = a.nstage - 1;
  uint32_t ph = 0;
  for (int64_t P = 0; P < npanel && !failed;
       ++P, stp = st, st = (st + 1 == a.nstage) ? 0 : st + 1, ph ^= (st == 0) ? 1u : 0u) {
    if (!mbar_wait_bounded(smem_u32(&mbar[st]), ph)) s_fail = 1;
    __syncthreads();
    if (s_fail) { failed = true; break; }
    // the previous panel's stage is free: refill it (the last warp issues the copies)
    if (tid == T - 32 && P >= 1 && P - 1 + a.nstage < npanel) issue1(P - 1 + a.nstage, stp);
    const CT* Ust = (const CT*)(stage0 + (size_t)st * stage_bytes);
    const CT* Uist = (const CT*)(stage0 + (size_t)st * stage_bytes + p1_cols);
    const int64_t j0 = P * NB;
    // head block: U_blk^H w_h = h, w_h[t] = sum_s conj(inv(U_blk)[s][t]) h[s], in NPART fixed
    // partial ranges of s (FP64: one warp each, then a barrier; FP32: all in one thread); the
    // head rows leave with w
    auto head_out = [&](int e, CT acc) {
      const int t = e / NC, c = e - (e / NC) * NC;
      xs[e] = acc;
      if (j0 + t < n && c < ncol) Yo[(int64_t)(c0 + c) * a.ldy + j0 + t] = acc;
    };
    if constexpr (sizeof(CT) == sizeof(float2)) {
      for (int e = tid; e < NB * NC; e += T) {
        const int t = e / NC, c = e - (e / NC) * NC;
        CT p[NPART];
#pragma unroll
        for (int g = 0; g < NPART; ++g) {
          p[g] = zero;
#pragma unroll
          for (int s2 = 2 * g; s2 < 2 * g + 2; ++s2)
            p[g] = cfma_conj(Uist[s2 * NB + t], hd[s2 * NC + c], p[g]);
        }
        head_out(e, sum_parts(p, 1, 0));
      }
    } else {
      for (int e = tid; e < NPART * NB * NC; e += T) {
        const int g = e / (NB * NC), o = e - g * (NB * NC);
        const int t = o / NC, c = o - (o / NC) * NC;
        CT acc = zero;
#pragma unroll
        for (int s2 = 2 * g; s2 < 2 * g + 2; ++s2)
          acc = cfma_conj(Uist[s2 * NB + t], hd[s2 * NC + c], acc);
        part[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < NB * NC; e += T) head_out(e, sum_parts(part, NB * NC, e));
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      const int s = tid + u * T;
      if (s >= Sf) continue;
      const int64_t r = row[u];
      const int base = (int)(r - j0);            // >= NB for every window row
#pragma unroll
      for (int jj = 0; jj < NB; ++jj) {
        const int d = base - jj;
        if (d <= kv) {
          const CT uu = Ust[(size_t)jj * kvp + d - 1];
#pragma unroll
          for (int c = 0; c < NC; ++c) v[u][c] = cfms_conj(uu, xs[jj * NC + c], v[u][c]);
        }
      }
      // rows j0+NB..j0+2NB-1 are the next panel's head: to hd, and the slot takes row r + Sf
      const int dh = base - NB;
      if (dh < NB) {
#pragma unroll
        for (int c = 0; c < NC; ++c) hd[dh * NC + c] = v[u][c];
        const int64_t r2 = r + Sf;
        row[u] = r2;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          v[u][c] = nxt[u][c];
          nxt[u][c] = (r2 + Sf < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + r2 + Sf] : zero;
        }
      }
    }
    __syncthreads();
  }
  __syncthreads();
  if (failed) {
    if (tid == 0) atomicExch(a.status + ST_TIMEOUT, 1);
    for (int st = 0; st < a.nstage; ++st)
      for (int ph = 0; ph < 2; ++ph) mbar_wait_bounded(smem_u32(&mbar[st]), (uint32_t)ph);
    return;
  }
  // re-initialise the barriers for phase 2 (every phase-1 stage has completed)
  if (tid == 0) {
    for (int i = 0; i < a.nstage; ++i) {
      mbar_inval(smem_u32(&mbar[i]));
      mbar_init(smem_u32(&mbar[i]), 1);
    }
    mbar_fence_init();
  }
  __syncthreads();

  // ------------------------------- phase 2: x = P^T L^{-H} w ----------------------------------
  // Descending blocks; window rows j0..j0+kl+7 in shared memory (slot = row mod S2).
  auto issue2 = [&](int64_t P, int st) {
    unsigned char* dst = stage0 + (size_t)st * stage_bytes;
    const uint32_t bar = smem_u32(&mbar[st]);
    mbar_expect_tx(bar, (uint32_t)p2_bytes);
    bulk_g2s(smem_u32(dst), Lp + P * NB * a.ldl, (uint32_t)p2_cols, bar);
    bulk_g2s(smem_u32(dst + p2_cols), Mp + P * (16 * MW), (uint32_t)(16 * MW * sizeof(CT)), bar);
    bulk_g2s(smem_u32(dst + p2_cols + 16 * MW * sizeof(CT)), Hp + P * 16,
             (uint32_t)(16 * sizeof(int)), bar);
  };
  if (tid == 0)
    for (int st = 0; st < a.nstage && st < npanel; ++st) issue2(npanel - 1 - st, st);
  {
    const int64_t jl = a.n_pad - NB;
    for (int e = tid; e < S2 * NC; e += T) {
      const int i = e / NC, c = e - (e / NC) * NC;
      const int64_t r = jl + i;
      win[(int)(r % S2) * NC + c] = (r < n && c < ncol) ? Yo[(int64_t)(c0 + c) * a.ldy + r] : zero;
    }
  }
  // the 8 rows entering the window at a panel's (C) are loaded one panel ahead, in registers
  // (NB * NC <= 64 <= 2 * T items, at most two per thread)
  CT pf[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int e = tid + i * T;
    pf[i] = zero;
    if (e < NB * NC) {
      const int t = e / NC, c = e - (e / NC) * NC;
      const int64_t r2 = a.n_pad - 2 * NB + t;
      if (r2 >= 0 && c < ncol) pf[i] = Yo[(int64_t)(c0 + c) * a.ldy + r2];
    }
  }
  // dot products: groups of g lanes (a power of two within a warp)
  int g = 32;
  while (g > 1 && g * NB * NC > T) g >>= 1;
  const int ngroups = T / g;
  __syncthreads();
  // window slot of the panel's first row j0 = (npanel-1-Bp)*NB, kept as a running counter:
  // slot(j0 + x) = s0 + x (- S2) for 0 <= x < 2*S2
  int s0 = (int)(((npanel - 1) * NB) % S2);
  auto slot = [&](int x) {
    const int sl = s0 + x;
    return sl >= S2 ? sl - S2 : sl;
  };
  st = 0;
  stp = a.nstage - 1;
  ph = 0;
  for (int64_t Bp = 0; Bp < npanel && !failed;
       ++Bp, stp = st, st = (st + 1 == a.nstage) ? 0 : st + 1, ph ^= (st == 0) ? 1u : 0u,
               s0 = (s0 - NB < 0) ? s0 - NB + S2 : s0 - NB) {
    const int64_t P = npanel - 1 - Bp;
    if (!mbar_wait_bounded(smem_u32(&mbar[st]), ph)) s_fail = 1;
    __syncthreads();
    if (s_fail) { failed = true; break; }
    if (tid == 0 && Bp >= 1 && Bp - 1 + a.nstage < npanel)
      issue2(npanel - 1 - (Bp - 1 + a.nstage), stp);
    const CT* Lst = (const CT*)(stage0 + (size_t)st * stage_bytes);
    const CT* Mst = (const CT*)(stage0 + (size_t)st * stage_bytes + p2_cols);
    const int* Hst = (const int*)(stage0 + (size_t)st * stage_bytes + p2_cols + 16 * MW * sizeof(CT));
    const int64_t j0 = P * NB;
    const int nvalid = (int)((n - j0) < NB ? (n - j0) : NB);
    // (A1) gather the members, mark the pivot members' slots
    for (int e = tid; e < 16 * NC; e += T) {
      const int m = e / NC, c = e - (e / NC) * NC;
      const int hr = Hst[m];
      hv[e] = (hr >= 0) ? win[slot(hr - (int)j0) * NC + c] : zero;
    }
    if (tid < NB && Hst[NB + tid] >= 0) mflag[slot(Hst[NB + tid] - (int)j0)] = 1;
    __syncthreads();
    // (A2) d_jj = sum over non-member rows r in (j, j+kl] of conj(L(r, j)) w_r
    for (int e0 = 0; e0 < NB * NC; e0 += ngroups) {
      const int e = e0 + tid / g, l = tid - (tid / g) * g;
      const bool act = (e < NB * NC) && (tid < ngroups * g);
      CT acc = zero;
      if (act) {
        const int jj = e / NC, c = e - (e / NC) * NC;
        if (jj < nvalid) {
          const int64_t j = j0 + jj;
          int sl = slot(jj + 1 + l);
          for (int i = l; i < kl; i += g) {
            const int64_t r = j + 1 + i;
            if (r >= n) break;
            if (r >= j0 + NB && !mflag[sl])
              acc = cfma_conj(Lst[(size_t)jj * klp + i], win[sl * NC + c], acc);
            sl += g;
            while (sl >= S2) sl -= S2;
          }
        }
      }
      for (int o = g / 2; o > 0; o >>= 1) acc = cadd_t(acc, shfl_xor_c(acc, o, g));
      if (act && l == 0) dv[e] = acc;
    }
    __syncthreads();
    // (B) H <- M1 H + M2 d
    for (int e = tid; e < 16 * NC; e += T) {
      const int m = e / NC, c = e - (e / NC) * NC;
      const int hr = Hst[m];
      if (hr < 0) continue;
      CT acc = zero;
#pragma unroll
      for (int m2 = 0; m2 < 16; ++m2) acc = cfma(Mst[m * MW + m2], hv[m2 * NC + c], acc);
#pragma unroll
      for (int jj = 0; jj < NB; ++jj) acc = cfma(Mst[m * MW + 16 + jj], dv[jj * NC + c], acc);
      win[slot(hr - (int)j0) * NC + c] = acc;
    }
    if (tid < NB && Hst[NB + tid] >= 0) mflag[slot(Hst[NB + tid] - (int)j0)] = 0;
    __syncthreads();
    // (C) rows j0+kl .. j0+kl+7 are final: write them; rows j0-8 .. j0-1 enter their slots
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int e = tid + i * T;
      if (e >= NB * NC) continue;
      const int t = e / NC, c = e - (e / NC) * NC;
      const int64_t r = j0 + kl + t;
      const int sl = slot(kl + t);
      if (r < n && c < ncol) out(r, c, win[sl * NC + c]);
      win[sl * NC + c] = pf[i];                       // row j0 - NB + t (zero if < 0)
      const int64_t r3 = j0 - 2 * NB + t;             // entering row of the next panel
      pf[i] = (r3 >= 0 && c < ncol) ? Yo[(int64_t)(c0 + c) * a.ldy + r3] : zero;
    }
    __syncthreads();
  }
  __syncthreads();
  if (failed) {
    if (tid == 0) atomicExch(a.status + ST_TIMEOUT, 1);
    for (int st = 0; st < a.nstage; ++st)
      for (int ph = 0; ph < 2; ++ph) mbar_wait_bounded(smem_u32(&mbar[st]), (uint32_t)ph);
    return;
  }
  // rows 0 .. kl-1 are still in the window
  for (int e = tid; e < kl * NC; e += T) {
    const int r = e / NC, c = e - (e / NC) * NC;
    if (r < n && c < ncol) out(r, c, win[(r % S2) * NC + c]);
  }
}

// ----------------------------------------------------------------------------------------------
template <typename CT, int NC, int SPT, int REGS>
static cudaError_t launch_adj_r(const AdjArgsT<CT>& a, int q, int threads, size_t smem,
                                cudaStream_t s) {
  auto kfn = band_solve_adj_kernel<CT, NC, SPT, REGS>;
  cudaError_t e = ie_smem_optin((const void*)kfn);
  if (e != cudaSuccess) return e;
  int blocks = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kfn, threads, smem);
  if (e != cudaSuccess) return e;
  if (blocks < 1) return cudaErrorLaunchOutOfResources;   // refuse rather than fail the launch
  dim3 grid((unsigned)((a.k + NC - 1) / NC), (unsigned)q);
  kfn<<<grid, threads, smem, s>>>(a); ie_count_launch();
  return cudaGetLastError();
}

// The register file is split over the SM's 4 sub-partitions (16K registers each): a block of
// W warps needs ceil(W/4) * 32 * REGS <= 16384, so 112 registers for <= 16 warps, else 96.
template <typename CT, int NC, int SPT>
static cudaError_t launch_adj_t(const AdjArgsT<CT>& a, int q, int threads, size_t smem,
                                cudaStream_t s) {
  if (threads <= 16 * 32) return launch_adj_r<CT, NC, SPT, 112>(a, q, threads, smem, s);
  return launch_adj_r<CT, NC, SPT, 96>(a, q, threads, smem, s);
}

template <typename CT>
static cudaError_t launch_adj(AdjArgsT<CT> a, int q, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const bool fp32 = sizeof(CT) == sizeof(float2);
  const int ncmax = fp32 ? 8 : 4;
  int nc = ncmax;
  for (int c = 1; c <= ncmax; c *= 2)
    if ((int64_t)q * ((a.k + c - 1) / c) <= sms) { nc = c; break; }
  const int slots = a.kv > NB ? a.kv : NB;   // phase-1 window (head rows in shared memory)
  const int spt = (slots > 576) ? 2 : 1;
  // two slots per thread with the widest column groups spill registers
  if (spt == 2) nc = std::min(nc, fp32 ? 4 : 2);
  if ((slots + spt - 1) / spt > 576) return cudaErrorInvalidValue;
  const int threads = ((slots + spt - 1) / spt + 31) / 32 * 32;
  const size_t p1 = (size_t)NB * a.kvp * sizeof(CT) + 64 * sizeof(CT);
  const size_t p2 = (size_t)NB * a.klp * sizeof(CT) + 16 * MW * sizeof(CT) + 16 * sizeof(int);
  const size_t stage_bytes = ((p1 > p2 ? p1 : p2) + 127) & ~(size_t)127;
  const size_t budget = 224 * 1024;   // below the 227 KB per-block opt-in limit
  auto fixed_for = [&](int c) {
    return 128 + (size_t)(3 * NB + 16 + NPART * NB) * c * sizeof(CT) +
           (size_t)(a.kl + NB) * c * sizeof(CT) +
           (size_t)(a.kl + NB) + 256;
  };
  while (nc > 1 && fixed_for(nc) + 2 * stage_bytes > budget) nc >>= 1;
  const size_t fixed = fixed_for(nc);
  if (fixed + 2 * stage_bytes > budget) return cudaErrorInvalidValue;
  int nstage = (int)((budget - fixed) / stage_bytes);
  if (nstage > 3) nstage = 3;
  a.nstage = nstage;
  const size_t smem = fixed + (size_t)nstage * stage_bytes;
#define IE_ADJ_CASE(NC_, SPT_) \
  if (nc == NC_ && spt == SPT_) return launch_adj_t<CT, NC_, SPT_>(a, q, threads, smem, s);
  IE_ADJ_CASE(1, 1) IE_ADJ_CASE(2, 1) IE_ADJ_CASE(4, 1)
  IE_ADJ_CASE(1, 2) IE_ADJ_CASE(2, 2) IE_ADJ_CASE(4, 2)
  if constexpr (sizeof(CT) == sizeof(float2)) {
    IE_ADJ_CASE(8, 1) IE_ADJ_CASE(8, 2)
  }
#undef IE_ADJ_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_band_solve_adj(int q, int64_t n, int kl, int64_t n_pad, const cplx* L64,
                                  const cplx* Ut64, const cplx* Ub, const cplx* M64, const int* Hb,
                                  const cplx* d_wconj, const cplx* RHS, int64_t ldr, int k,
                                  cplx* Xp, int64_t ldx, int64_t xstride, int* status,
                                  cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  AdjArgsT<cplx> a{};
  a.n = n; a.n_pad = n_pad; a.kl = kl; a.kv = 2 * kl; a.klp = kl; a.kvp = 2 * kl; a.k = k;
  a.mode = 0;
  a.L = L64; a.ldl = kl; a.lstride = n_pad * kl;
  a.Ut = Ut64; a.ldu = 2 * kl; a.ustride = n_pad * 2 * kl;
  a.Ub = Ub; a.Mb = M64; a.Hb = Hb; a.weights = d_wconj;
  a.RHS = RHS; a.ldr = ldr; a.rstride = 0;
  a.Y = Xp; a.ldy = ldx; a.ystride = xstride;
  a.X = Xp; a.ldx = ldx; a.xstride = xstride;
  a.status = status;
  return launch_adj(a, q, s);
}

cudaError_t launch_band_solve_adj32(int q, int64_t n, int kl, int64_t n_pad, const float2* L32,
                                    int64_t ldl, const float2* Ut32, const float2* Ui32,
                                    const float2* M32, const int* Hb, const cplx* d_wconj,
                                    const float2* RHS, int64_t ldr, int64_t rstride, int k,
                                    float2* Y32, int64_t ldy, int64_t ystride, cplx* X,
                                    int64_t ldx, int64_t xstride, int accumulate, int* status,
                                    cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  AdjArgsT<float2> a{};
  a.n = n; a.n_pad = n_pad; a.kl = kl; a.kv = 2 * kl; a.klp = (int)ldl; a.kvp = 2 * kl;
  a.k = k; a.mode = accumulate ? 3 : 1;
  a.L = L32; a.ldl = ldl; a.lstride = n_pad * ldl;
  a.Ut = Ut32; a.ldu = 2 * kl; a.ustride = n_pad * 2 * kl;
  a.Ub = Ui32; a.Mb = M32; a.Hb = Hb; a.weights = d_wconj;
  a.RHS = RHS; a.ldr = ldr; a.rstride = rstride;
  a.Y = Y32; a.ldy = ldy; a.ystride = ystride;
  a.X = X; a.ldx = ldx; a.xstride = xstride;
  a.status = status;
  return launch_adj(a, q, s);
}

// ----------------------------------------------------------------------------------------------
// Sensitivities of simple eigenvalues to the diagonal of A (first-order perturbation theory):
//   den_i = y_i^H B x_i,  S[j, i] = alpha conj(y_i[j]) x_i[j] / den_i,
//   grad[j] = Re sum_i conj(gbar_i) S[j, i].
// One CTA per column for den (deterministic order), then one thread per row j.
__global__ void coldot_kernel(int64_t n, const cplx* Y, int64_t ldy, const cplx* BX, int64_t ldb,
                              cplx* den) {
  const int i = blockIdx.x;
  const cplx* y = Y + (int64_t)i * ldy;
  const cplx* bx = BX + (int64_t)i * ldb;
  cplx acc = make_double2(0, 0);
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) acc = cfma_conj(y[j], bx[j], acc);
  __shared__ cplx red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    cplx t = make_double2(0, 0);
    for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) t = cadd(t, red[wv]);
    den[i] = t;
  }
}

__global__ void sensitivity_kernel(int64_t n, int nf, const cplx* X, int64_t ldx, const cplx* Y,
                                   int64_t ldy, const cplx* den, cplx alpha, cplx* S, int64_t lds,
                                   const cplx* gbar, double* grad) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  double gsum = 0.0;
  for (int i = 0; i < nf; ++i) {
    const cplx sij = cdiv(cmul(alpha, cmul(cconj(Y[(int64_t)i * ldy + j]), X[(int64_t)i * ldx + j])), den[i]);
    if (S) S[(int64_t)i * lds + j] = sij;
    if (grad) gsum += gbar[i].x * sij.x + gbar[i].y * sij.y;   // Re(conj(gbar) s)
  }
  if (grad) grad[j] = gsum;
}

void launch_sensitivity(const DiaDev& P, int nf, const cplx* X, int64_t ldx, const cplx* Y,
                        int64_t ldy, cplx alpha, cplx* BX, cplx* den, cplx* S, int64_t lds,
                        const cplx* gbar, double* grad, cudaStream_t s) {
  if (nf <= 0) return;
  launch_spmv(P, make_double2(0, 0), make_double2(1, 0), X, ldx, nullptr, nf, BX, P.n, s);
  coldot_kernel<<<nf, 256, 0, s>>>(P.n, Y, ldy, BX, P.n, den); ie_count_launch();
  sensitivity_kernel<<<(unsigned)((P.n + 255) / 256), 256, 0, s>>>(P.n, nf, X, ldx, Y, ldy, den,
                                                                   alpha, S, lds, gbar, grad); ie_count_launch();
}

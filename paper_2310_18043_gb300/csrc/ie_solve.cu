// Band triangular solves of the inner operator G (Sec. 3.2, Eq. linearsolve2):
// x_i = K_i^{-1} rhs with K_i = P_i^T L_i U_i from the batched band LU, for all q poles and
// k right-hand sides in one launch. Complex128 (the plain path) or complex64 factors with
// FP32 arithmetic (the mixed-precision path, refined in FP64 by the caller).
//
// One CTA per (pole, group of NC right-hand sides): the row recurrence is sequential in n,
// so parallelism comes from poles x column groups and from the band width inside each step.
// Forward sweep (P, L; LAPACK zgbtrs order: swap, then eliminate): the window of S = kl+1 rows
// j..j+kl lives in registers, one row slot per thread (slot = row mod S); per row the pivot
// values are broadcast through a double-buffered shared cell, one barrier per row.
// Backward sweep (U), blocked: one block = one staged panel of NB columns; the NB head rows
// are solved by NC threads (a small triangular solve), then every slot applies the NB columns
// at once; two barriers per NB rows.
// Factor columns (L parts forward, U parts backward, with pivots / 1/u_jj) are staged NB at a
// time into a shared ring by cp.async.bulk (TMA bulk copies) with mbarrier completion; every
// wait is bounded.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ie_internal.cuh"
#include "ie_bulk.cuh"

using namespace iebulk;

namespace {
constexpr int NB = 8;   // factor columns per staged panel = backward block
}  // namespace

template <typename CT>
struct SolveArgsT {
  int64_t n, n_pad;
  int kl, kv, klp, kvp, k, nstage, mode;
  // factors, split and contiguous: column col's L part (kl entries, padded to klp) at
  // L + pole*lstride + col*ldl with ldl = klp, U part (rows col-kv..col-1, kvp = kv entries)
  // at U + pole*ustride + col*ldu with ldu = kvp
  const CT* L;
  const CT* U;
  int64_t ldl, ldu, lstride, ustride;
  const int* piv;     // 0-based, pole stride n_pad
  const CT* dinv;     // 1/u_jj, pole stride n_pad
  // per (pole, panel) block transforms (see block_transform_kernel): forward 16x16 T and its
  // member rows, backward 8x8 inverse of U's diagonal block
  const CT* Tb;       // [pole][panel][16][16], column m of T at m*16
  const int* Hb;      // [pole][panel][16]
  const CT* Ub;       // [pole][panel][8][8]
  const cplx* weights;
  const CT* RHS;      // column c at RHS + pole*rstride + c*ldr
  int64_t ldr, rstride;
  CT* Y;              // forward result, column c at Y + pole*ystride + c*ldy
  int64_t ldy, ystride;
  cplx* X;            // output (mode 0: X == Y, X = w*x; mode 1: X = x; mode 3: x written in
                      // place into Y in the element type, X untouched)
  int64_t ldx, xstride;
  int* status;
};

// REGS: register budget. The register file is split over the SM's 4 sub-partitions (16K
// registers each) and a block's warps are spread over them, so a block of W warps needs
// ceil(W/4) * 32 * REGS <= 16384: 112 registers allow 16 warps, 96 allow 20.
//
// Window layout. The rows a panel's columns update are held in registers, one row per slot
// (SPT slots per thread); the NB head rows being solved live in shared memory (hd). Forward:
// the panel with head rows j0..j0+NB-1 updates rows j0+NB..j0+NB+kl-1, so the window has
// Sf = max(kl, NB) slots (slot = (row - NB) mod Sf). Backward: the panel with head rows
// j0-NB+1..j0 updates rows j0-NB-kv+1..j0-NB, so Sb = max(kv, NB) slots (slot =
// (n_pad-1-NB - row) mod Sb). After a panel's update the window's NB rows nearest the head
// become the next head: they move to hd and their slots take the rows entering the window
// (S rows further on, not yet touched by any solved column). Keeping the head out of the
// register window makes the thread count S / SPT (a multiple of 4 warps for kl = 256 or
// 512), so every sub-partition of the SM gets the same share of the update.
// Bit m set: member m of the panel's set H is present (H entry >= 0).
__device__ __forceinline__ unsigned present_mask(const int* Hst) {
  const int4* h4 = reinterpret_cast<const int4*>(Hst);   // 16-byte aligned in every stage
  unsigned pres = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int4 t = h4[k];
    pres |= ((t.x >= 0 ? 1u : 0u) | (t.y >= 0 ? 2u : 0u) | (t.z >= 0 ? 4u : 0u) |
             (t.w >= 0 ? 8u : 0u)) << (4 * k);
  }
  return pres;
}
// the NC values of one head output row (NC even, complex64: 16-byte loads)
template <typename CT, int NC>
__device__ __forceinline__ void ld_row(const CT* p, CT (&o)[NC]) {
  if constexpr (sizeof(CT) == sizeof(float2) && NC % 2 == 0) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int k = 0; k < NC / 2; ++k) {
      const float4 t = q[k];
      o[2 * k] = make_float2(t.x, t.y);
      o[2 * k + 1] = make_float2(t.z, t.w);
    }
  } else {
#pragma unroll
    for (int k = 0; k < NC; ++k) o[k] = p[k];
  }
}
// One window row's forward update by a panel's NB columns: row j0 + dr (dr >= NB) minus
// L(row, j0+jj) * y_jj over the columns jj < nvalid whose band reaches the row (dd = dr - jj
// <= kl). Every load is unconditional (out-of-band entries read a valid word and use zero), so
// the loads of all NB columns can be in flight together.
template <typename CT, int NC>
__device__ __forceinline__ void fwd_update(CT (&v)[NC], const CT* Lst, const CT* hv2, int dr,
                                           int nvalid, int kl, int klp) {
  const CT zero{};
#pragma unroll
  for (int jj = 0; jj < NB; ++jj) {
    const int dd = dr - jj;                  // dd >= NB - jj >= 1 for every window row
    const bool inb = jj < nvalid && dd <= kl;
    const CT l0 = Lst[jj * klp + (inb ? dd - 1 : 0)];
    const CT lv = inb ? l0 : zero;
    CT x[NC];
    ld_row<CT, NC>(hv2 + jj * NC, x);
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = cfms(lv, x[c], v[c]);
  }
}
// One window row's backward update: row j0 - base (base >= NB) minus U(row, j0-s2) * x_s2 for
// the panel's columns j0-s2 with d = base - s2 <= kv, loads unconditional as above.
template <typename CT, int NC>
__device__ __forceinline__ void bwd_update(CT (&v)[NC], const CT* Ust, const CT* xs, int base,
                                           int kv, int kvp) {
  const CT zero{};
#pragma unroll
  for (int s2 = 0; s2 < NB; ++s2) {
    const int d = base - s2;                 // d >= NB - s2 >= 1
    const bool inb = d <= kv;
    const CT u0 = Ust[(NB - 1 - s2) * kvp + (inb ? kv - d : 0)];
    const CT uu = inb ? u0 : zero;
    CT x[NC];
    ld_row<CT, NC>(xs + s2 * NC, x);
#pragma unroll
    for (int c = 0; c < NC; ++c) v[c] = cfms(uu, x[c], v[c]);
  }
}

// One CTA's work: pole `pole`, right-hand sides grp*NC .. grp*NC+NC-1 of the solve `a`.
template <typename CT, int NC, int SPT>
__device__ __forceinline__ void solve_cta(const SolveArgsT<CT>& a, const int pole, const int grp) {
  const int c0 = grp * NC;
  const int ncol = min(NC, a.k - c0);
  const int T = blockDim.x, tid = threadIdx.x;
  const int kl = a.kl, kv = a.kv, klp = a.klp, kvp = a.kvp;
  const int64_t n = a.n;
  const CT* Lp = a.L + (int64_t)pole * a.lstride;
  const CT* Up = a.U + (int64_t)pole * a.ustride;
  const int64_t npan = a.n_pad / NB;
  const CT* Tp = a.Tb + (int64_t)pole * npan * 256;
  const int* Hp = a.Hb + (int64_t)pole * npan * 16;
  const CT* Uip = a.Ub + (int64_t)pole * npan * 64;
  const CT* R = a.RHS + (int64_t)pole * a.rstride;
  CT* Yo = a.Y + (int64_t)pole * a.ystride;
  cplx* Xo = a.X + (int64_t)pole * a.xstride;
  const cplx w = a.weights[pole];
  const CT zero{};

  extern __shared__ __align__(128) unsigned char sm_raw[];
  uint64_t* mbar = (uint64_t*)sm_raw;                          // nstage mbarriers
  CT* hd = (CT*)(sm_raw + 128);                                // [NB][NC] head values
  CT* xs = hd + NB * NC;                                       // [NB][NC] solved head
  CT* hv = xs + NB * NC;                                       // [16][NC] forward set H
  CT* hv2 = hv + 16 * NC;                                      // [16][NC] T H
  CT* part = hv2 + 16 * NC;                                    // [NPART][16][NC] partials
  unsigned char* stage0 =
      (unsigned char*)(((uintptr_t)(part + NPART * 16 * NC) + 127) & ~(uintptr_t)127);
  const size_t fwd_cols_bytes = (size_t)NB * klp * sizeof(CT);
  const size_t bwd_cols_bytes = (size_t)NB * kvp * sizeof(CT);
  const size_t fwd_bytes = fwd_cols_bytes + 256 * sizeof(CT) + 16 * sizeof(int);
  const size_t bwd_bytes = bwd_cols_bytes + 64 * sizeof(CT);
  const size_t stage_bytes = ((fwd_bytes > bwd_bytes ? fwd_bytes : bwd_bytes) + 127) & ~(size_t)127;
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
  // the last warp issues the bulk copies, so that warp 0 (head solves) never waits on it
  const int issuer = T - 32;

  if (tid == 0) {
    s_fail = 0;
    for (int i = 0; i < a.nstage; ++i) mbar_init(smem_u32(&mbar[i]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();

  const int64_t npanel = a.n_pad / NB;
  // ------------------------------- forward: P L y = rhs -------------------------------------
  // Panel P, steps j0..j0+NB-1 (j0 = P*NB). Only the NB head rows and the panel's pivot rows
  // take part in swaps; on that set H (16 members) the panel's swaps and eliminations are the
  // fixed 16x16 matrix T (precomputed from the factors), so: (A) gather H (head rows from hd,
  // pivot members from the window), (B) H <- T H in parallel, the head rows leave with y,
  // (C) pivot members take their values, every other window row applies the panel's NB
  // multipliers at once, and the window's first NB rows move to hd. Three barriers per panel.
  auto issue_fwd = [&](int64_t P, int st) {
    unsigned char* dst = stage0 + (size_t)st * stage_bytes;
    const uint32_t bar = smem_u32(&mbar[st]);
    mbar_expect_tx(bar, (uint32_t)(fwd_cols_bytes + 256 * sizeof(CT) + 16 * sizeof(int)));
    // the panel's NB columns are contiguous (ldl = klp): one copy
    bulk_g2s(smem_u32(dst), Lp + P * NB * a.ldl, (uint32_t)fwd_cols_bytes, bar);
    bulk_g2s(smem_u32(dst + fwd_cols_bytes), Tp + P * 256, (uint32_t)(256 * sizeof(CT)), bar);
    bulk_g2s(smem_u32(dst + fwd_cols_bytes + 256 * sizeof(CT)), Hp + P * 16,
             (uint32_t)(16 * sizeof(int)), bar);
  };
  const int Sf = kl > NB ? kl : NB;
  CT v[SPT][NC], nxt[SPT][NC];
  int64_t frow[SPT];
  if (tid == issuer)
    for (int st = 0; st < a.nstage && st < npanel; ++st) issue_fwd(st, st);
  for (int e = tid; e < NB * NC; e += T) {
    const int t = e / NC, c = e - (e / NC) * NC;
    hd[e] = (t < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + t] : zero;
  }
#pragma unroll
  for (int u = 0; u < SPT; ++u) {
    const int s = tid + u * T;
    const int64_t r = NB + s;
    frow[u] = r;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      v[u][c] = (s < Sf && r < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + r] : zero;
      nxt[u][c] = (s < Sf && r + Sf < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + r + Sf] : zero;
    }
  }
  bool failed = false;
  // stage ring position and mbarrier phase of the current panel, kept as running 32-bit
  // counters (a 64-bit division by the runtime stage count per panel costs more than the
  // panel's own bookkeeping)
  int st = 0, stp = a.nstage - 1;
  uint32_t ph = 0;
  for (int64_t P = 0; P < npanel && !failed;
       ++P, stp = st, st = (st + 1 == a.nstage) ? 0 : st + 1, ph ^= (st == 0) ? 1u : 0u) {
    if (!mbar_wait_bounded(smem_u32(&mbar[st]), ph)) s_fail = 1;
    __syncthreads();
    if (s_fail) { failed = true; break; }
    // the previous panel's stage is free: refill it
    if (tid == issuer && P >= 1 && P - 1 + a.nstage < npanel) issue_fwd(P - 1 + a.nstage, stp);
    const CT* Lst = (const CT*)(stage0 + (size_t)st * stage_bytes);
    const CT* Tst = (const CT*)(stage0 + (size_t)st * stage_bytes + fwd_cols_bytes);
    const int* Hst = (const int*)(stage0 + (size_t)st * stage_bytes + fwd_cols_bytes + 256 * sizeof(CT));
    const int64_t j0 = P * NB;
    const int nvalid = (int)((n - j0) < NB ? (n - j0) : NB);
    // (A) gather: head rows from hd, pivot members (H entries NB..15) from the window; absent
    // members are zero (their column of T is zero too)
    for (int e = tid; e < NB * NC; e += T) {
      hv[e] = hd[e];
      if (Hst[NB + e / NC] < 0) hv[NB * NC + e] = zero;
    }
    int mem[SPT];
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      const int s = tid + u * T;
      mem[u] = -1;
      if (s >= Sf) continue;
      const int dr = (int)(frow[u] - j0);   // row offset from the panel head (32-bit)
      const int j0i = (int)j0;
#pragma unroll
      for (int i = NB; i < 16; ++i)
        if (Hst[i] - j0i == dr) mem[u] = i;
      if (mem[u] >= 0)
#pragma unroll
        for (int c = 0; c < NC; ++c) hv[mem[u] * NC + c] = v[u][c];
    }
    __syncthreads();
    // (B) H <- T H in NPART partial sums, then their fixed-order sum; the head rows' results
    // are final: y. FP64: the partials on consecutive warps (spread over the SM
    // sub-partitions, whose FP64 units are the bound), one more barrier; FP32: one thread
    // computes all partials of its output (latency, not throughput, bounds this step).
    if constexpr (sizeof(CT) == sizeof(float2)) {
      const unsigned pres = present_mask(Hst);
      for (int e = tid; e < 16 * NC; e += T) {
        const int i = e / NC, c = e - (e / NC) * NC;
        if ((pres >> i) & 1u) {
          CT p[NPART];
#pragma unroll
          for (int g = 0; g < NPART; ++g) {
            p[g] = zero;
#pragma unroll
            for (int m = 4 * g; m < 4 * g + 4; ++m)
              p[g] = cfma(Tst[m * 16 + i], hv[m * NC + c], p[g]);
          }
          const CT acc = sum_parts(p, 1, 0);
          hv2[e] = acc;
          if (i < nvalid && c < ncol) Yo[(int64_t)(c0 + c) * a.ldy + j0 + i] = acc;
        }
      }
      __syncthreads();
    } else {
    for (int e = tid; e < NPART * 16 * NC; e += T) {
      const int g = e / (16 * NC), o = e - g * (16 * NC);
      const int i = o / NC, c = o - (o / NC) * NC;
      CT acc = zero;
      if (Hst[i] >= 0) {
#pragma unroll
        for (int m = 4 * g; m < 4 * g + 4; ++m)
          if (Hst[m] >= 0) acc = cfma(Tst[m * 16 + i], hv[m * NC + c], acc);
      }
      part[e] = acc;
    }
    __syncthreads();
    for (int e = tid; e < 16 * NC; e += T) {
      const int i = e / NC, c = e - (e / NC) * NC;
      if (Hst[i] >= 0) {
        const CT acc = sum_parts(part, 16 * NC, e);
        hv2[e] = acc;
        if (i < nvalid && c < ncol) Yo[(int64_t)(c0 + c) * a.ldy + j0 + i] = acc;
      }
    }
    __syncthreads();
    }
    // (C)
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      const int s = tid + u * T;
      if (s >= Sf) continue;
      const int64_t r = frow[u];
      const int i = mem[u];
      fwd_update<CT, NC>(v[u], Lst, hv2, (int)(r - j0), nvalid, kl, klp);
      if (i >= NB) {
#pragma unroll
        for (int c = 0; c < NC; ++c) v[u][c] = hv2[i * NC + c];
      }
      // rows j0+NB..j0+2NB-1 are the next panel's head: to hd, and the slot takes row r + Sf
      const int dh = (int)(r - j0) - NB;
      if (dh < NB) {
#pragma unroll
        for (int c = 0; c < NC; ++c) hd[dh * NC + c] = v[u][c];
        const int64_t r2 = r + Sf;
        frow[u] = r2;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          v[u][c] = nxt[u][c];
          nxt[u][c] = (r2 + Sf < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + r2 + Sf] : zero;
        }
      }
    }
  }
  __syncthreads();
  if (failed) {
    if (tid == 0) atomicExch(a.status + ST_TIMEOUT, 1);
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
  // ------------------------------- backward: U x = y (blocked) -------------------------------
  // Panel Bp, head rows j0-NB+1..j0 (j0 = n_pad - 1 - Bp*NB) in hd (hd[t] = row j0 - t); the
  // window holds rows j0-NB-Sb+1..j0-NB. Rows >= n are virtual: zero values, zero factor
  // columns, zero 1/u_jj. x_head = inv(U_block) h_head, then every window row applies the
  // panel's NB columns; the window's first NB rows move to hd. Two barriers per panel.
  auto issue_bwd = [&](int64_t Bp, int st) {
    unsigned char* dst = stage0 + (size_t)st * stage_bytes;
    const uint32_t bar = smem_u32(&mbar[st]);
    const int64_t cb0 = a.n_pad - (Bp + 1) * NB;
    mbar_expect_tx(bar, (uint32_t)(bwd_cols_bytes + 64 * sizeof(CT)));
    bulk_g2s(smem_u32(dst), Up + cb0 * a.ldu, (uint32_t)bwd_cols_bytes, bar);   // contiguous
    bulk_g2s(smem_u32(dst + bwd_cols_bytes), Uip + (cb0 / NB) * 64, (uint32_t)(64 * sizeof(CT)),
             bar);
  };
  const int Sb = kv > NB ? kv : NB;
  int64_t row[SPT];
  if (tid == issuer)
    for (int st = 0; st < a.nstage && st < npanel; ++st) issue_bwd(st, st);
  {
    const int64_t j0 = a.n_pad - 1;
    for (int e = tid; e < NB * NC; e += T) {
      const int t = e / NC, c = e - (e / NC) * NC;
      const int64_t r = j0 - t;
      hd[e] = (r < n && c < ncol) ? Yo[(int64_t)(c0 + c) * a.ldy + r] : zero;
    }
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      const int s = tid + u * T;
      const int64_t r = j0 - NB - s;
      row[u] = r;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        v[u][c] = (s < Sb && r >= 0 && r < n && c < ncol) ? Yo[(int64_t)(c0 + c) * a.ldy + r] : zero;
        const int64_t rn = r - Sb;
        nxt[u][c] = (s < Sb && rn >= 0 && rn < n && c < ncol) ? Yo[(int64_t)(c0 + c) * a.ldy + rn]
                                                             : zero;
      }
    }
  }
  st = 0;
  stp = a.nstage - 1;
  ph = 0;
  for (int64_t Bp = 0; Bp < npanel && !failed;
       ++Bp, stp = st, st = (st + 1 == a.nstage) ? 0 : st + 1, ph ^= (st == 0) ? 1u : 0u) {
    if (!mbar_wait_bounded(smem_u32(&mbar[st]), ph)) s_fail = 1;
    __syncthreads();
    if (s_fail) { failed = true; break; }
    // the previous panel's stage is free: refill it
    if (tid == issuer && Bp >= 1 && Bp - 1 + a.nstage < npanel) issue_bwd(Bp - 1 + a.nstage, stp);
    const CT* Ust = (const CT*)(stage0 + (size_t)st * stage_bytes);
    const CT* Uist = (const CT*)(stage0 + (size_t)st * stage_bytes + bwd_cols_bytes);
    const int64_t j0 = a.n_pad - 1 - Bp * NB;
    // head rows j0 - t (t = 0..NB-1) = block rows NB-1-t; matrix column j0 - s2 is stage
    // column NB-1-s2. x_head = inv(U_block) h_head in NPART partial sums over the head rows
    // (FP64: one warp each for NC = 4, then a barrier; FP32: all in one thread), then their
    // fixed-order sum; the head rows leave with x
    auto head_out = [&](int e, CT acc) {
      const int t = e / NC, c = e - (e / NC) * NC;
      xs[t * NC + c] = acc;
      const int64_t r = j0 - t;
      if (r < n && c < ncol) {
        if constexpr (sizeof(CT) == sizeof(cplx)) {
          if (a.mode == 0) Yo[(int64_t)(c0 + c) * a.ldy + r] = cmul(w, acc);
        }
        if (a.mode == 1) Xo[(int64_t)(c0 + c) * a.ldx + r] = to_d(acc);
        else if (a.mode == 3) Yo[(int64_t)(c0 + c) * a.ldy + r] = acc;   // y of row r is read
      }
    };
    if constexpr (sizeof(CT) == sizeof(float2)) {
      for (int e = tid; e < NB * NC; e += T) {
        const int t = e / NC, c = e - (e / NC) * NC;
        CT p[NPART];
#pragma unroll
        for (int g = 0; g < NPART; ++g) {
          p[g] = zero;
#pragma unroll
          for (int t2 = 2 * g; t2 < 2 * g + 2; ++t2)
            p[g] = cfma(Uist[(NB - 1 - t) * NB + (NB - 1 - t2)], hd[t2 * NC + c], p[g]);
        }
        head_out(e, sum_parts(p, 1, 0));
      }
    } else {
      for (int e = tid; e < NPART * NB * NC; e += T) {
        const int g = e / (NB * NC), o = e - g * (NB * NC);
        const int t = o / NC, c = o - (o / NC) * NC;
        CT acc = zero;
#pragma unroll
        for (int t2 = 2 * g; t2 < 2 * g + 2; ++t2)
          acc = cfma(Uist[(NB - 1 - t) * NB + (NB - 1 - t2)], hd[t2 * NC + c], acc);
        part[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < NB * NC; e += T) head_out(e, sum_parts(part, NB * NC, e));
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      const int s = tid + u * T;
      if (s >= Sb) continue;
      const int64_t r = row[u];
      const int base = (int)(j0 - r);            // >= NB for every window row
      bwd_update<CT, NC>(v[u], Ust, xs, base, kv, kvp);
      // rows j0-NB..j0-2NB+1 are the next panel's head: to hd, and the slot takes row r - Sb
      const int dh = base - NB;
      if (dh < NB) {
#pragma unroll
        for (int c = 0; c < NC; ++c) hd[dh * NC + c] = v[u][c];
        const int64_t r2 = r - Sb;
        row[u] = r2;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          v[u][c] = nxt[u][c];
          const int64_t rn = r2 - Sb;
          nxt[u][c] = (rn >= 0 && rn < n && c < ncol) ? Yo[(int64_t)(c0 + c) * a.ldy + rn] : zero;
        }
      }
    }
  }
  __syncthreads();
  if (failed) {
    if (tid == 0) atomicExch(a.status + ST_TIMEOUT, 1);
    for (int st = 0; st < a.nstage; ++st)
      for (int ph = 0; ph < 2; ++ph) mbar_wait_bounded(smem_u32(&mbar[st]), (uint32_t)ph);
  }
}

template <typename CT, int NC, int SPT, int REGS>
__global__ void __maxnreg__(REGS) band_solve_kernel(SolveArgsT<CT> a) {
  solve_cta<CT, NC, SPT>(a, blockIdx.y, blockIdx.x);
}

// Many independent solves (different problems: n, band, poles, block width, factors) in one
// launch. CTA b serves solve cta[b].x, pole cta[b].y, column group cta[b].z; the block size is
// that of the widest band, and each solve's window uses its own slot count. Every CTA's
// arithmetic is that of band_solve_kernel for its solve.
template <typename CT, int NC, int SPT, int REGS>
__global__ void __maxnreg__(REGS) band_solve_batch_kernel(const SolveArgsT<CT>* items,
                                                          const int4* cta) {
  const int4 m = cta[blockIdx.x];
  const SolveArgsT<CT> a = items[m.x];
  solve_cta<CT, NC, SPT>(a, m.y, m.z);
}

// ----------------------------------------------------------------------------------------------
// Warp-specialised form of the same solve: no CTA-wide barrier per panel.
//
// Roles: warps 0..WU-1 hold the register window (as above, slot = tid + u*WU*32); warp WU is
// the head warp (the forward H <- T H and the backward x_head = inv(U_block) h_head, and the
// head rows' global outputs); warp WU+1 is the producer (bulk copies of the factor panels).
// The two sweeps are one sequence of 2*npanel panels G (forward P = G, backward Bp =
// G - npanel) sharing a ring of ns stages. Stage G % ns holds the factor panel (bulk copy),
// the head warp's output OUT (forward: T H, 16 x NC; backward: x_head, NB x NC) and its input
// IN (forward: the 16 members; backward: the NB head rows). Per stage four mbarriers:
//   FULL  (bulk copy landed; count 1 + tx bytes),
//   EMPTY (every update warp and the head warp are done with the stage; count WU + 1),
//   HDF   (IN complete; count 2*NB: one arrival per head row from the update thread that holds
//          it, one per present pivot member (forward), the rest by the head warp),
//   XSF   (OUT complete; count 1, the head warp).
// An update thread whose row becomes a head row of panel G+1 writes it into IN(G+1) and
// arrives on HDF(G+1) as soon as its own update of panel G is done, so the head warp starts
// panel G+1 while other rows are still being updated with panel G. Every barrier of panel G
// waits behind FULL(G), and FULL(G) behind EMPTY(G - ns), so no warp runs ns panels ahead of
// another and no mbarrier phase is passed twice unseen. The in-place output of the backward
// sweep (mode 0/3) is safe: a row's y is loaded by the thread that later hands the row to
// the head warp. Every wait is bounded; on a timeout the CTA records ST_TIMEOUT, every warp
// leaves its loop, and the producer waits for the bulk copies it issued before exiting.
namespace {
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_cnt(uint32_t bar, uint32_t cnt) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(cnt) : "memory");
}
// bounded wait that also gives up when another warp has recorded a failure; a timeout is
// recorded in the CTA's flag and in the kernel's status word
__device__ __forceinline__ bool pwait(uint32_t bar, uint32_t parity, volatile int* fail,
                                      int* status) {
  if (mbar_try_wait_sleep(bar, parity, IE_SUSPEND_NS)) return true;
  const unsigned long long t0 = ie_globaltimer();
  while (true) {
    if (mbar_try_wait_sleep(bar, parity, IE_SUSPEND_NS)) return true;
    if (*fail) return false;
    if (ie_globaltimer() - t0 > IE_WAIT_NS) {
      *fail = 1;
      atomicExch(status + ST_TIMEOUT, 1);
      return false;
    }
  }
}
}  // namespace

template <typename CT, int NC, int SPT, int REGS>
__global__ void __maxnreg__(REGS) band_solve_pipe_kernel(SolveArgsT<CT> a) {
  const int pole = blockIdx.y;
  const int c0 = blockIdx.x * NC;
  const int ncol = min(NC, a.k - c0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int WU = (int)(blockDim.x >> 5) - 2;      // update warps
  const int TU = WU * 32;                         // update threads
  const int kl = a.kl, kv = a.kv, klp = a.klp, kvp = a.kvp;
  const int64_t n = a.n;
  const CT* Lp = a.L + (int64_t)pole * a.lstride;
  const CT* Up = a.U + (int64_t)pole * a.ustride;
  const int64_t npan = a.n_pad / NB;
  const CT* Tp = a.Tb + (int64_t)pole * npan * 256;
  const int* Hp = a.Hb + (int64_t)pole * npan * 16;
  const CT* Uip = a.Ub + (int64_t)pole * npan * 64;
  const CT* R = a.RHS + (int64_t)pole * a.rstride;
  CT* Yo = a.Y + (int64_t)pole * a.ystride;
  cplx* Xo = a.X + (int64_t)pole * a.xstride;
  const cplx w = a.weights[pole];
  const CT zero{};
  const int ns = a.nstage;
  const int64_t npanel = npan, total = 2 * npan;

  extern __shared__ __align__(128) unsigned char sm_raw[];
  uint64_t* bars = (uint64_t*)sm_raw;             // [4][ns]: FULL, EMPTY, HDF, XSF
  const size_t fwd_cols_bytes = (size_t)NB * klp * sizeof(CT);
  const size_t bwd_cols_bytes = (size_t)NB * kvp * sizeof(CT);
  const size_t fwd_bytes = fwd_cols_bytes + 256 * sizeof(CT) + 16 * sizeof(int);
  const size_t bwd_bytes = bwd_cols_bytes + 64 * sizeof(CT);
  const size_t fac_bytes = ((fwd_bytes > bwd_bytes ? fwd_bytes : bwd_bytes) + 127) & ~(size_t)127;
  const size_t io_bytes = (size_t)16 * NC * sizeof(CT);
  const size_t stage_bytes = (fac_bytes + 2 * io_bytes + 127) & ~(size_t)127;
  unsigned char* stage0 = sm_raw + ((4 * (size_t)ns * 8 + 127) & ~(size_t)127);
  __shared__ int s_fail_raw;
  volatile int* s_fail = &s_fail_raw;
  {
    unsigned dsz;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsz));
    if ((size_t)(stage0 - sm_raw) + (size_t)ns * stage_bytes > (size_t)dsz || WU < 1 ||
        (ns != 2 && ns != 4)) {
      if (tid == 0) atomicExch(a.status + ST_TIMEOUT, 1);
      return;
    }
  }
  // ns is 2 or 4 (the host sizes it so): stage = G mod ns and phase = (G div ns) mod 2 by masks
  // and shifts, not by a division per use
  const int lgns = ns == 4 ? 2 : 1;
  auto sidx = [&](int64_t G) { return (int)(G & (ns - 1)); };
  auto FULL = [&](int64_t G) { return smem_u32(&bars[0 * ns + sidx(G)]); };
  auto EMPTY = [&](int64_t G) { return smem_u32(&bars[1 * ns + sidx(G)]); };
  auto HDF = [&](int64_t G) { return smem_u32(&bars[2 * ns + sidx(G)]); };
  auto XSF = [&](int64_t G) { return smem_u32(&bars[3 * ns + sidx(G)]); };
  auto par = [&](int64_t G) { return (uint32_t)((G >> lgns) & 1); };
  auto FAC = [&](int64_t G) { return stage0 + (size_t)sidx(G) * stage_bytes; };
  auto OUT = [&](int64_t G) { return (CT*)(stage0 + (size_t)sidx(G) * stage_bytes + fac_bytes); };
  auto IN = [&](int64_t G) {
    return (CT*)(stage0 + (size_t)sidx(G) * stage_bytes + fac_bytes + io_bytes);
  };
  if (tid == 0) {
    s_fail_raw = 0;
    for (int i = 0; i < ns; ++i) {
      mbar_init(smem_u32(&bars[0 * ns + i]), 1);
      mbar_init(smem_u32(&bars[1 * ns + i]), (uint32_t)(WU + 1));
      mbar_init(smem_u32(&bars[2 * ns + i]), 2 * NB);
      mbar_init(smem_u32(&bars[3 * ns + i]), 1);
    }
    mbar_fence_init();
  }
  __syncthreads();

  const int Sf = kl > NB ? kl : NB;
  const int Sb = kv > NB ? kv : NB;
  // ---------------------------------------------------------------- producer warp
  auto issue = [&](int64_t G) {
    unsigned char* dst = FAC(G);
    const uint32_t bar = FULL(G);
    if (G < npanel) {
      const int64_t P = G;
      mbar_expect_tx(bar, (uint32_t)fwd_bytes);
      bulk_g2s(smem_u32(dst), Lp + P * NB * a.ldl, (uint32_t)fwd_cols_bytes, bar);
      bulk_g2s(smem_u32(dst + fwd_cols_bytes), Tp + P * 256, (uint32_t)(256 * sizeof(CT)), bar);
      bulk_g2s(smem_u32(dst + fwd_cols_bytes + 256 * sizeof(CT)), Hp + P * 16,
               (uint32_t)(16 * sizeof(int)), bar);
    } else {
      const int64_t cb0 = a.n_pad - (G - npanel + 1) * NB;
      mbar_expect_tx(bar, (uint32_t)bwd_bytes);
      bulk_g2s(smem_u32(dst), Up + cb0 * a.ldu, (uint32_t)bwd_cols_bytes, bar);
      bulk_g2s(smem_u32(dst + bwd_cols_bytes), Uip + (cb0 / NB) * 64, (uint32_t)(64 * sizeof(CT)),
               bar);
    }
  };
  int64_t issued = 0;
  auto produce_until = [&](int64_t Gend) {   // lane 0 of the producer warp
    for (; issued < Gend && !*s_fail; ++issued) {
      if (issued >= ns && !pwait(EMPTY(issued - ns), par(issued - ns), s_fail, a.status)) break;
      issue(issued);
    }
  };
  auto drain = [&]() {   // wait for the bulk copies still in flight (bounded)
    for (int64_t G = issued - ns > 0 ? issued - ns : 0; G < issued; ++G)
      if (!mbar_wait_bounded(FULL(G), par(G))) atomicExch(a.status + ST_TIMEOUT, 1);
  };
  const bool is_prod = warp == WU + 1, is_head = warp == WU;

  // ---------------------------------------------------------------- forward sweep
  CT v[SPT][NC], nxt[SPT][NC];
  int64_t frow[SPT];
  int mem[SPT];
  if (is_prod) {
    if (lane == 0) {
      produce_until(npanel + ns < total ? npanel + ns : total);
      if (*s_fail) drain();
    }
  } else if (is_head) {
    // panel 0's head rows come from the right-hand side; the head warp also completes the
    // HDF count of every forward panel for the pivot members that are absent
    for (int e = lane; e < NB * NC; e += 32) {
      const int t = e / NC, c = e - (e / NC) * NC;
      IN(0)[t * NC + c] = (t < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + t] : zero;
    }
    __syncwarp();
    if (lane == 0) mbar_arrive_cnt(HDF(0), NB);
    for (int64_t P = 0; P < npanel; ++P) {
      const int64_t G = P;
      if (!pwait(FULL(G), par(G), s_fail, a.status)) break;
      const unsigned char* st = FAC(G);
      const CT* Tst = (const CT*)(st + fwd_cols_bytes);
      const int* Hst = (const int*)(st + fwd_cols_bytes + 256 * sizeof(CT));
      const unsigned pres = present_mask(Hst);
      const int npres = __popc(pres >> NB);
      // absent members take the value zero: their column of T is zero too, so the products
      // below can run over all 16 members unconditionally and still equal the sums over the
      // present ones (a partial starts at +0 and so never becomes -0)
      for (int e = lane; e < NB * NC; e += 32)
        if (!((pres >> (NB + e / NC)) & 1u)) IN(G)[NB * NC + e] = zero;
      __syncwarp();
      if (lane == 0 && npres < NB) mbar_arrive_cnt(HDF(G), (uint32_t)(NB - npres));
      if (!pwait(HDF(G), par(G), s_fail, a.status)) break;
      const CT* hv = IN(G);
      CT* hv2 = OUT(G);
      const int64_t j0 = P * NB;
      const int nvalid = (int)((n - j0) < NB ? (n - j0) : NB);
      // lanes 16h..16h+15 take the 16 outputs of one column: the reads of one T column are 16
      // consecutive words, and no load waits behind a branch
      constexpr int NE = (16 * NC + 31) / 32;
#pragma unroll
      for (int it = 0; it < NE; ++it) {
        const int e = lane + 32 * it;
        const int i = e & 15, c = e >> 4;
        if (c < NC) {
          CT p[NPART];
#pragma unroll
          for (int g = 0; g < NPART; ++g) {
            p[g] = zero;
#pragma unroll
            for (int m = 4 * g; m < 4 * g + 4; ++m)
              p[g] = cfma(Tst[m * 16 + i], hv[m * NC + c], p[g]);
          }
          const CT acc = sum_parts(p, 1, 0);
          if ((pres >> i) & 1u) {
            hv2[i * NC + c] = acc;
            if (i < nvalid && c < ncol) Yo[(int64_t)(c0 + c) * a.ldy + j0 + i] = acc;
          }
        }
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(XSF(G));
        mbar_arrive(EMPTY(G));
      }
    }
  } else {
    // update warps: initial window rows NB.. and panel 0's pivot members
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      const int s = tid + u * TU;
      const int64_t r = NB + s;
      frow[u] = r;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        v[u][c] = (s < Sf && r < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + r] : zero;
        nxt[u][c] = (s < Sf && r + Sf < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + r + Sf] : zero;
      }
    }
    // member index of each slot for panel P (H entries NB..15), and hand the members over
    auto members = [&](int64_t P) -> bool {
      const int64_t G = P;
      if (!pwait(FULL(G), par(G), s_fail, a.status)) return false;
      const int* Hst = (const int*)(FAC(G) + fwd_cols_bytes + 256 * sizeof(CT));
      CT* hv = IN(G);
      const int j0i = (int)(P * NB);
#pragma unroll
      for (int u = 0; u < SPT; ++u) {
        const int s = tid + u * TU;
        mem[u] = -1;
        if (s >= Sf) continue;
        const int dr = (int)(frow[u] - P * NB);
#pragma unroll
        for (int i = NB; i < 16; ++i)
          if (Hst[i] - j0i == dr) mem[u] = i;
        if (mem[u] >= 0) {
#pragma unroll
          for (int c = 0; c < NC; ++c) hv[mem[u] * NC + c] = v[u][c];
          mbar_arrive(HDF(G));
        }
      }
      return true;
    };
    bool ok = members(0);
    for (int64_t P = 0; P < npanel && ok; ++P) {
      const int64_t G = P;
      if (!pwait(XSF(G), par(G), s_fail, a.status)) break;   // FULL(G) was waited on by members(P)
      const unsigned char* st = FAC(G);
      const CT* Lst = (const CT*)st;
      const CT* hv2 = OUT(G);
      const int64_t j0 = P * NB;
      const int nvalid = (int)((n - j0) < NB ? (n - j0) : NB);
      const bool more = P + 1 < npanel;
      CT* hdn = more ? IN(G + 1) : nullptr;
#pragma unroll
      for (int u = 0; u < SPT; ++u) {
        const int s = tid + u * TU;
        if (s >= Sf) continue;
        const int64_t r = frow[u];
        const int i = mem[u];
        fwd_update<CT, NC>(v[u], Lst, hv2, (int)(r - j0), nvalid, kl, klp);
        if (i >= NB) {
#pragma unroll
          for (int c = 0; c < NC; ++c) v[u][c] = hv2[i * NC + c];
        }
        const int dh = (int)(r - j0) - NB;
        if (dh < NB) {   // a head row of panel P+1: hand it over, take row r + Sf
          if (more) {
#pragma unroll
            for (int c = 0; c < NC; ++c) hdn[dh * NC + c] = v[u][c];
            mbar_arrive(HDF(G + 1));
          }
          const int64_t r2 = r + Sf;
          frow[u] = r2;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            v[u][c] = nxt[u][c];
            nxt[u][c] = (r2 + Sf < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + r2 + Sf] : zero;
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(EMPTY(G));
      if (more && !members(P + 1)) break;
    }
  }
  // the forward results y (written by the head warp) are read back by every warp below
  __syncthreads();

  // ---------------------------------------------------------------- backward sweep
  if (!*s_fail) {
    if (is_prod) {
      if (lane == 0) {
        produce_until(total);
        // stay until every stage has been consumed, so that no bulk copy can outlive the CTA
        for (int64_t G = total - ns > 0 ? total - ns : 0; G < total && !*s_fail; ++G)
          pwait(EMPTY(G), par(G), s_fail, a.status);
        if (*s_fail) drain();
      }
    } else if (is_head) {
      {
        const int64_t j0 = a.n_pad - 1;
        CT* hd = IN(npanel);
        for (int e = lane; e < NB * NC; e += 32) {
          const int t = e / NC, c = e - (e / NC) * NC;
          const int64_t r = j0 - t;
          hd[e] = (r < n && c < ncol) ? Yo[(int64_t)(c0 + c) * a.ldy + r] : zero;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive_cnt(HDF(npanel), NB);
      }
      for (int64_t Bp = 0; Bp < npanel; ++Bp) {
        const int64_t G = npanel + Bp;
        if (!pwait(FULL(G), par(G), s_fail, a.status)) break;
        if (lane == 0) mbar_arrive_cnt(HDF(G), NB);
        if (!pwait(HDF(G), par(G), s_fail, a.status)) break;
        const CT* Uist = (const CT*)(FAC(G) + bwd_cols_bytes);
        const CT* hd = IN(G);
        CT* xs = OUT(G);
        const int64_t j0 = a.n_pad - 1 - Bp * NB;
        for (int e = lane; e < NB * NC; e += 32) {
          const int t = e / NC, c = e - (e / NC) * NC;
          CT p[NPART];
#pragma unroll
          for (int g = 0; g < NPART; ++g) {
            p[g] = zero;
#pragma unroll
            for (int t2 = 2 * g; t2 < 2 * g + 2; ++t2)
              p[g] = cfma(Uist[(NB - 1 - t) * NB + (NB - 1 - t2)], hd[t2 * NC + c], p[g]);
          }
          const CT acc = sum_parts(p, 1, 0);
          xs[t * NC + c] = acc;
          const int64_t r = j0 - t;
          if (r < n && c < ncol) {
            if constexpr (sizeof(CT) == sizeof(cplx)) {
              if (a.mode == 0) Yo[(int64_t)(c0 + c) * a.ldy + r] = cmul(w, acc);
            }
            if (a.mode == 1) Xo[(int64_t)(c0 + c) * a.ldx + r] = to_d(acc);
            else if (a.mode == 3) Yo[(int64_t)(c0 + c) * a.ldy + r] = acc;
          }
        }
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(XSF(G));
          mbar_arrive(EMPTY(G));
        }
      }
    } else {
      int64_t row[SPT];
      {
        const int64_t j0 = a.n_pad - 1;
#pragma unroll
        for (int u = 0; u < SPT; ++u) {
          const int s = tid + u * TU;
          const int64_t r = j0 - NB - s;
          row[u] = r;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            v[u][c] = (s < Sb && r >= 0 && r < n && c < ncol) ? Yo[(int64_t)(c0 + c) * a.ldy + r] : zero;
            const int64_t rn = r - Sb;
            nxt[u][c] = (s < Sb && rn >= 0 && rn < n && c < ncol) ? Yo[(int64_t)(c0 + c) * a.ldy + rn]
                                                                 : zero;
          }
        }
      }
      for (int64_t Bp = 0; Bp < npanel; ++Bp) {
        const int64_t G = npanel + Bp;
        if (!pwait(FULL(G), par(G), s_fail, a.status)) break;
        if (!pwait(XSF(G), par(G), s_fail, a.status)) break;
        const CT* Ust = (const CT*)FAC(G);
        const CT* xs = OUT(G);
        const int64_t j0 = a.n_pad - 1 - Bp * NB;
        const bool more = Bp + 1 < npanel;
        CT* hdn = more ? IN(G + 1) : nullptr;
#pragma unroll
        for (int u = 0; u < SPT; ++u) {
          const int s = tid + u * TU;
          if (s >= Sb) continue;
          const int64_t r = row[u];
          const int base = (int)(j0 - r);
          bwd_update<CT, NC>(v[u], Ust, xs, base, kv, kvp);
          const int dh = base - NB;
          if (dh < NB) {
            if (more) {
#pragma unroll
              for (int c = 0; c < NC; ++c) hdn[dh * NC + c] = v[u][c];
              mbar_arrive(HDF(G + 1));
            }
            const int64_t r2 = r - Sb;
            row[u] = r2;
#pragma unroll
            for (int c = 0; c < NC; ++c) {
              v[u][c] = nxt[u][c];
              const int64_t rn = r2 - Sb;
              nxt[u][c] = (rn >= 0 && rn < n && c < ncol) ? Yo[(int64_t)(c0 + c) * a.ldy + rn] : zero;
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(EMPTY(G));
      }
    }
  }
}

// ----------------------------------------------------------------------------------------------
// Look-ahead warp-specialised kernel. The chain that bounds the kernels above is, per panel,
// head product -> update of the rows that form the next head -> next head product: the
// warps holding those rows finish their whole update before the head can go on. Here the
// update warps run one panel behind the head instead:
//  * at panel P the update warps apply P to the window as before, and then hand the head
//    warps the values, after panel P, of the rows panel P+2 needs (its head rows and pivot
//    members; a member may also sit in a slot's next row, not yet in the window);
//  * the head warps of panel P+2 apply panel P+1 to those 16 rows themselves (the same
//    operations, in the same order, as the update warps apply to them, so the values are
//    identical), take the rows that were members of P+1 from their own output, and form
//    H <- T H.
// The head warps thus never wait for an update of the current panel; the update warps have a
// whole panel of slack. NH = NC/2 head warps take two right-hand sides each (no exchange
// between them: every step of the head is per column). Stage G of the ring holds the factor
// panel (forward: L columns, T, H(G) and H(G+2), the member set two panels on; backward: U
// columns, inv(U_block)), OUT(G) (forward: T H; backward: x_head) and IN(G) (the rows the head
// of G needs, after panel G-2). Per stage four mbarriers:
//   FULL  (bulk copy landed; count 1 + tx bytes),
//   EMPTY (every update warp is done with the stage, and every head warp with it and with the
//          catch-up of the next panel; count WU + NH),
//   HDF   (IN complete; count 2*NB: one arrival per delivered row, the rest by head warp 0),
//   XSF   (OUT complete; count NH).
// Panels 0 and 1 of each sweep read their inputs directly (no panel before them has touched
// them). The update warps write IN(G+2) while processing G (after head G): the stage's
// previous use G+2-ns was last read by head G+2-ns (IN) and head G+3-ns (factors and OUT of
// the catch-up), both before head G for ns >= 3, and the update warps still reading OUT(G-1)
// for ns = 3 touch another part of the stage. Every wait is bounded.
// One CTA's work: pole `pole`, right-hand sides grp*NC .. grp*NC+NC-1 of the solve `a`.
template <typename CT, int NC, int SPT>
__device__ __forceinline__ void la_cta(const SolveArgsT<CT>& a, const int pole, const int grp) {
  constexpr int HC = NC >= 2 ? 2 : 1;          // right-hand sides per head warp
  constexpr int NH = NC / HC;                  // head warps
  const int c0 = grp * NC;
  const int ncol = min(NC, a.k - c0);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int WU = (int)(blockDim.x >> 5) - NH - 1;   // update warps
  const int TU = WU * 32;
  const int kl = a.kl, kv = a.kv, klp = a.klp, kvp = a.kvp;
  const int64_t n = a.n;
  const CT* Lp = a.L + (int64_t)pole * a.lstride;
  const CT* Up = a.U + (int64_t)pole * a.ustride;
  const int64_t npan = a.n_pad / NB;
  const CT* Tp = a.Tb + (int64_t)pole * npan * 256;
  const int* Hp = a.Hb + (int64_t)pole * npan * 16;
  const CT* Uip = a.Ub + (int64_t)pole * npan * 64;
  const CT* R = a.RHS + (int64_t)pole * a.rstride;
  CT* Yo = a.Y + (int64_t)pole * a.ystride;
  cplx* Xo = a.X + (int64_t)pole * a.xstride;
  const cplx w = a.weights[pole];
  const CT zero{};
  const int ns = a.nstage;
  const int64_t npanel = npan, total = 2 * npan;

  extern __shared__ __align__(128) unsigned char sm_raw[];
  uint64_t* bars = (uint64_t*)sm_raw;             // [4][ns]: FULL, EMPTY, HDF, XSF
  const size_t fwd_cols_bytes = (size_t)NB * klp * sizeof(CT);
  const size_t bwd_cols_bytes = (size_t)NB * kvp * sizeof(CT);
  const size_t fwd_bytes = fwd_cols_bytes + 256 * sizeof(CT) + 32 * sizeof(int);
  const size_t bwd_bytes = bwd_cols_bytes + 64 * sizeof(CT);
  const size_t fac_bytes = ((fwd_bytes > bwd_bytes ? fwd_bytes : bwd_bytes) + 127) & ~(size_t)127;
  const size_t io_bytes = (size_t)16 * NC * sizeof(CT);
  const size_t stage_bytes = (fac_bytes + 2 * io_bytes + 127) & ~(size_t)127;
  unsigned char* stage0 = sm_raw + ((4 * (size_t)ns * 8 + 127) & ~(size_t)127);
  __shared__ int s_fail_raw;
  volatile int* s_fail = &s_fail_raw;
  {
    unsigned dsz;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(dsz));
    if ((size_t)(stage0 - sm_raw) + (size_t)ns * stage_bytes > (size_t)dsz || WU < 1 || ns < 3) {
      if (tid == 0) atomicExch(a.status + ST_TIMEOUT, 1);
      return;
    }
  }
  auto FULL = [&](int s) { return smem_u32(&bars[0 * ns + s]); };
  auto EMPTY = [&](int s) { return smem_u32(&bars[1 * ns + s]); };
  auto HDF = [&](int s) { return smem_u32(&bars[2 * ns + s]); };
  auto XSF = [&](int s) { return smem_u32(&bars[3 * ns + s]); };
  auto FAC = [&](int s) { return stage0 + (size_t)s * stage_bytes; };
  auto OUT = [&](int s) { return (CT*)(stage0 + (size_t)s * stage_bytes + fac_bytes); };
  auto IN = [&](int s) { return (CT*)(stage0 + (size_t)s * stage_bytes + fac_bytes + io_bytes); };
  auto HS = [&](int s) { return (const int*)(FAC(s) + fwd_cols_bytes + 256 * sizeof(CT)); };
  auto HS2 = [&](int s) { return HS(s) + 16; };
  // ring position of a panel as running counters: stage s (G mod ns) and parity ph
  auto advance = [&](int& s, uint32_t& ph) {
    if (++s == ns) { s = 0; ph ^= 1u; }
  };
  auto plus = [&](int s, int d) { return s + d >= ns ? s + d - ns : s + d; };   // 0 <= d < ns
  auto minus1 = [&](int s) { return s == 0 ? ns - 1 : s - 1; };
  if (tid == 0) {
    s_fail_raw = 0;
    for (int i = 0; i < ns; ++i) {
      mbar_init(FULL(i), 1);
      mbar_init(EMPTY(i), (uint32_t)(WU + NH));
      mbar_init(HDF(i), 2 * NB);
      mbar_init(XSF(i), (uint32_t)NH);
    }
    mbar_fence_init();
  }
  __syncthreads();

  const int Sf = kl > 2 * NB ? kl : 2 * NB;    // forward window (two heads ahead must fit)
  const int Sb = kv > 2 * NB ? kv : 2 * NB;
  const bool is_prod = warp == WU + NH, is_head = warp >= WU && warp < WU + NH;
  const int hw = warp - WU;                    // head warp index
  // ---------------------------------------------------------------- producer warp
  int p_s = 0;
  uint32_t p_ph = 0;
  int64_t issued = 0;
  auto issue = [&](int64_t G, int s) {
    unsigned char* dst = FAC(s);
    const uint32_t bar = FULL(s);
    if (G < npanel) {
      const int64_t P = G;
      const bool h2 = P + 2 < npanel;
      mbar_expect_tx(bar, (uint32_t)(fwd_cols_bytes + 256 * sizeof(CT) + (h2 ? 32 : 16) * sizeof(int)));
      bulk_g2s(smem_u32(dst), Lp + P * NB * a.ldl, (uint32_t)fwd_cols_bytes, bar);
      bulk_g2s(smem_u32(dst + fwd_cols_bytes), Tp + P * 256, (uint32_t)(256 * sizeof(CT)), bar);
      bulk_g2s(smem_u32(dst + fwd_cols_bytes + 256 * sizeof(CT)), Hp + P * 16,
               (uint32_t)(16 * sizeof(int)), bar);
      if (h2)
        bulk_g2s(smem_u32(dst + fwd_cols_bytes + 256 * sizeof(CT) + 16 * sizeof(int)),
                 Hp + (P + 2) * 16, (uint32_t)(16 * sizeof(int)), bar);
    } else {
      const int64_t cb0 = a.n_pad - (G - npanel + 1) * NB;
      mbar_expect_tx(bar, (uint32_t)bwd_bytes);
      bulk_g2s(smem_u32(dst), Up + cb0 * a.ldu, (uint32_t)bwd_cols_bytes, bar);
      bulk_g2s(smem_u32(dst + bwd_cols_bytes), Uip + (cb0 / NB) * 64, (uint32_t)(64 * sizeof(CT)),
               bar);
    }
  };
  auto produce_until = [&](int64_t Gend) {   // lane 0 of the producer warp
    for (; issued < Gend && !*s_fail; ++issued, advance(p_s, p_ph)) {
      if (issued >= ns && !pwait(EMPTY(p_s), p_ph ^ 1u, s_fail, a.status)) break;
      issue(issued, p_s);
    }
  };
  auto drain = [&]() {   // wait for the bulk copies still in flight (bounded)
    int s = p_s;
    uint32_t ph = p_ph;
    for (int64_t G = issued - 1; G >= 0 && G >= issued - ns; --G) {
      if (s == 0) { s = ns - 1; ph ^= 1u; } else { --s; }
      if (!mbar_wait_bounded(FULL(s), ph)) atomicExch(a.status + ST_TIMEOUT, 1);
    }
  };

  CT v[SPT][NC], nxt[SPT][NC];
  int64_t frow[SPT];
  // the update warps' ring position (both sweeps)
  int u_s = 0;
  uint32_t u_ph = 0;
  // the head warps' ring position
  int h_s = 0;
  uint32_t h_ph = 0;
  // ---------------------------------------------------------------- forward sweep
  if (is_prod) {
    if (lane == 0) produce_until(npanel + ns < total ? npanel + ns : total);
  } else if (is_head) {
    // lane -> (member i, right-hand side c): 16 lanes per column, HC columns per warp
    const int i = lane & 15, cc = lane >> 4, c = hw * HC + cc;
    const bool act = cc < HC;
    for (int64_t P = 0; P < npanel; ++P, advance(h_s, h_ph)) {
      const int s = h_s;
      if (!pwait(FULL(s), h_ph, s_fail, a.status)) break;
      const int* H = HS(s);
      const unsigned pres = present_mask(H);
      CT* in = IN(s);
      if (P < 2) {
        // no panel has touched these rows yet: read them from the right-hand side
        if (act) {
          const int r = H[i];
          in[i * NC + c] = (r >= 0 && r < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + r] : zero;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive_cnt(HDF(s), hw == 0 ? (uint32_t)(2 * NB - (NH - 1)) : 1u);
      } else if (hw == 0 && lane == 0) {
        const int npres = __popc(pres >> NB);
        if (npres < NB) mbar_arrive_cnt(HDF(s), (uint32_t)(NB - npres));
      }
      if (!pwait(HDF(s), h_ph, s_fail, a.status)) break;
      const int64_t j0 = P * NB;
      const int nvalid = (int)((n - j0) < NB ? (n - j0) : NB);
      // catch-up: the members after panel P-1 (IN holds them after panel P-2); members of
      // panel P-1 take its output, the others apply its NB columns as the update warps do
      if (act) {
        const int r = H[i];
        CT val = zero;
        if (r >= 0) {
          val = in[i * NC + c];
          if (P >= 1) {
            const int sp = minus1(s);
            const int* Hq = HS(sp);
            const CT* oq = OUT(sp);
            int idx = -1;
#pragma unroll
            for (int m = NB; m < 16; ++m)
              if (Hq[m] == r) idx = m;
            if (idx >= 0) {
              val = oq[idx * NC + c];
            } else {
              const CT* Lq = (const CT*)FAC(sp);
              const int64_t jq = j0 - NB;
              const int nvq = (int)((n - jq) < NB ? (n - jq) : NB);
              const int dr = (int)(r - jq);
#pragma unroll
              for (int jj = 0; jj < NB; ++jj) {
                const int dd = dr - jj;
                const bool inb = jj < nvq && dd <= kl;
                const CT l0 = Lq[jj * klp + (inb ? dd - 1 : 0)];
                val = cfms(inb ? l0 : zero, oq[jj * NC + c], val);
              }
            }
          }
        }
        in[i * NC + c] = val;
      }
      __syncwarp();
      // H <- T H
      if (act) {
        const CT* Tst = (const CT*)(FAC(s) + fwd_cols_bytes);
        CT p[NPART];
#pragma unroll
        for (int g = 0; g < NPART; ++g) {
          p[g] = zero;
#pragma unroll
          for (int m = 4 * g; m < 4 * g + 4; ++m) p[g] = cfma(Tst[m * 16 + i], in[m * NC + c], p[g]);
        }
        const CT acc = sum_parts(p, 1, 0);
        if ((pres >> i) & 1u) {
          OUT(s)[i * NC + c] = acc;
          if (i < nvalid && c < ncol) Yo[(int64_t)(c0 + c) * a.ldy + j0 + i] = acc;
        }
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(XSF(s));
        if (P >= 1) mbar_arrive(EMPTY(minus1(s)));   // panel P-1's factors and output
      }
    }
    if (!*s_fail && lane == 0 && npanel > 0) mbar_arrive(EMPTY(minus1(h_s)));
  } else {
    // update warps: window rows NB + slot, next rows NB + slot + Sf
#pragma unroll
    for (int u = 0; u < SPT; ++u) {
      const int sl = tid + u * TU;
      const int64_t r = NB + sl;
      frow[u] = r;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        v[u][c] = (sl < Sf && r < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + r] : zero;
        nxt[u][c] = (sl < Sf && r + Sf < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + r + Sf] : zero;
      }
    }
    for (int64_t P = 0; P < npanel; ++P, advance(u_s, u_ph)) {
      const int s = u_s;
      if (!pwait(FULL(s), u_ph, s_fail, a.status)) break;
      if (!pwait(XSF(s), u_ph, s_fail, a.status)) break;
      const CT* Lst = (const CT*)FAC(s);
      const int* H = HS(s);
      const int* H2 = HS2(s);
      const CT* hv2 = OUT(s);
      const int64_t j0 = P * NB;
      const int nvalid = (int)((n - j0) < NB ? (n - j0) : NB);
      const bool deliver = P + 2 < npanel;
      const int s2 = plus(s, 2);
      CT* in2 = IN(s2);
      int hm[NB], h2m[NB];
#pragma unroll
      for (int m = 0; m < NB; ++m) {
        hm[m] = H[NB + m];
        h2m[m] = deliver ? H2[NB + m] : -1;
      }
#pragma unroll
      for (int u = 0; u < SPT; ++u) {
        const int sl = tid + u * TU;
        if (sl >= Sf) continue;
        const int64_t r = frow[u];
        const int ri = (int)r;
        const int dr = (int)(r - j0);
        fwd_update<CT, NC>(v[u], Lst, hv2, dr, nvalid, kl, klp);
        int mem = -1;
#pragma unroll
        for (int m = 0; m < NB; ++m)
          if (hm[m] == ri) mem = NB + m;
        if (mem >= 0) {
#pragma unroll
          for (int c = 0; c < NC; ++c) v[u][c] = hv2[mem * NC + c];
        }
        if (deliver) {
          // rows of panel P+2's set: its head rows, members in this row or in the next row
          const int d2 = dr - 2 * NB;
          if (d2 >= 0 && d2 < NB) {
#pragma unroll
            for (int c = 0; c < NC; ++c) in2[d2 * NC + c] = v[u][c];
            mbar_arrive(HDF(s2));
          }
          int mv = -1, mn = -1;
#pragma unroll
          for (int m = 0; m < NB; ++m) {
            if (h2m[m] == ri) mv = NB + m;
            if (h2m[m] == ri + Sf) mn = NB + m;
          }
          if (mv >= 0) {
#pragma unroll
            for (int c = 0; c < NC; ++c) in2[mv * NC + c] = v[u][c];
            mbar_arrive(HDF(s2));
          }
          if (mn >= 0) {
#pragma unroll
            for (int c = 0; c < NC; ++c) in2[mn * NC + c] = nxt[u][c];
            mbar_arrive(HDF(s2));
          }
        }
        if (dr - NB < NB) {   // a head row of panel P+1 (the head warps finish it): take r + Sf
          const int64_t r2 = r + Sf;
          frow[u] = r2;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            v[u][c] = nxt[u][c];
            nxt[u][c] = (r2 + Sf < n && c < ncol) ? R[(int64_t)(c0 + c) * a.ldr + r2 + Sf] : zero;
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(EMPTY(s));
    }
  }
  // the forward results y (written by the head warps) are read back by every warp below
  __syncthreads();

  // ---------------------------------------------------------------- backward sweep
  if (*s_fail) {
    if (is_prod && lane == 0) drain();
    return;
  }
  if (is_prod) {
    if (lane == 0) {
      produce_until(total);
      // stay until every stage has been consumed, so that no bulk copy can outlive the CTA
      int s = p_s;
      uint32_t ph = p_ph;
      for (int64_t G = total - 1; G >= 0 && G >= total - ns && !*s_fail; --G) {
        if (s == 0) { s = ns - 1; ph ^= 1u; } else { --s; }
        pwait(EMPTY(s), ph, s_fail, a.status);
      }
      if (*s_fail) drain();
    }
  } else if (is_head) {
    // lane -> (head row t, right-hand side c): 8 lanes per column
    const int t = lane & 7, cc = lane >> 3, c = hw * HC + cc;
    const bool act = cc < HC;
    for (int64_t Bp = 0; Bp < npanel; ++Bp, advance(h_s, h_ph)) {
      const int s = h_s;
      if (!pwait(FULL(s), h_ph, s_fail, a.status)) break;
      const int64_t j0 = a.n_pad - 1 - Bp * NB;
      CT* in = IN(s);
      if (Bp < 2) {
        if (act) {
          const int64_t r = j0 - t;
          in[t * NC + c] = (r < n && c < ncol) ? Yo[(int64_t)(c0 + c) * a.ldy + r] : zero;
        }
        __syncwarp();
        if (lane == 0) mbar_arrive_cnt(HDF(s), hw == 0 ? (uint32_t)(2 * NB - (NH - 1)) : 1u);
      } else if (hw == 0 && lane == 0) {
        mbar_arrive_cnt(HDF(s), NB);
      }
      if (!pwait(HDF(s), h_ph, s_fail, a.status)) break;
      // catch-up: the head rows after panel Bp-1, from their values after panel Bp-2
      if (act) {
        CT val = in[t * NC + c];
        if (Bp >= 1) {
          const int sp = minus1(s);
          const CT* Uq = (const CT*)FAC(sp);
          const CT* xq = OUT(sp);
          const int base = NB + t;
#pragma unroll
          for (int s2 = 0; s2 < NB; ++s2) {
            const int d = base - s2;
            const bool inb = d <= kv;
            const CT u0 = Uq[(NB - 1 - s2) * kvp + (inb ? kv - d : 0)];
            val = cfms(inb ? u0 : zero, xq[s2 * NC + c], val);
          }
        }
        in[t * NC + c] = val;
      }
      __syncwarp();
      if (act) {
        const CT* Uist = (const CT*)(FAC(s) + bwd_cols_bytes);
        CT p[NPART];
#pragma unroll
        for (int g = 0; g < NPART; ++g) {
          p[g] = zero;
#pragma unroll
          for (int t2 = 2 * g; t2 < 2 * g + 2; ++t2)
            p[g] = cfma(Uist[(NB - 1 - t) * NB + (NB - 1 - t2)], in[t2 * NC + c], p[g]);
        }
        const CT acc = sum_parts(p, 1, 0);
        OUT(s)[t * NC + c] = acc;
        const int64_t r = j0 - t;
        if (r < n && c < ncol) {
          if constexpr (sizeof(CT) == sizeof(cplx)) {
            if (a.mode == 0) Yo[(int64_t)(c0 + c) * a.ldy + r] = cmul(w, acc);
          }
          if (a.mode == 1) Xo[(int64_t)(c0 + c) * a.ldx + r] = to_d(acc);
          else if (a.mode == 3) Yo[(int64_t)(c0 + c) * a.ldy + r] = acc;
        }
      }
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(XSF(s));
        if (Bp >= 1) mbar_arrive(EMPTY(minus1(s)));
      }
    }
    if (!*s_fail && lane == 0 && npanel > 0) mbar_arrive(EMPTY(minus1(h_s)));
  } else {
    int64_t row[SPT];
    {
      const int64_t j0 = a.n_pad - 1;
#pragma unroll
      for (int u = 0; u < SPT; ++u) {
        const int sl = tid + u * TU;
        const int64_t r = j0 - NB - sl;
        row[u] = r;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          v[u][c] = (sl < Sb && r >= 0 && r < n && c < ncol) ? Yo[(int64_t)(c0 + c) * a.ldy + r] : zero;
          const int64_t rn = r - Sb;
          nxt[u][c] = (sl < Sb && rn >= 0 && rn < n && c < ncol) ? Yo[(int64_t)(c0 + c) * a.ldy + rn]
                                                                : zero;
        }
      }
    }
    for (int64_t Bp = 0; Bp < npanel; ++Bp, advance(u_s, u_ph)) {
      const int s = u_s;
      if (!pwait(FULL(s), u_ph, s_fail, a.status)) break;
      if (!pwait(XSF(s), u_ph, s_fail, a.status)) break;
      const CT* Ust = (const CT*)FAC(s);
      const CT* xs = OUT(s);
      const int64_t j0 = a.n_pad - 1 - Bp * NB;
      const bool deliver = Bp + 2 < npanel;
      const int s2 = plus(s, 2);
      CT* in2 = IN(s2);
#pragma unroll
      for (int u = 0; u < SPT; ++u) {
        const int sl = tid + u * TU;
        if (sl >= Sb) continue;
        const int64_t r = row[u];
        const int base = (int)(j0 - r);
        bwd_update<CT, NC>(v[u], Ust, xs, base, kv, kvp);
        const int t2 = base - 2 * NB;   // a head row of panel Bp+2
        if (deliver && t2 >= 0 && t2 < NB) {
#pragma unroll
          for (int c = 0; c < NC; ++c) in2[t2 * NC + c] = v[u][c];
          mbar_arrive(HDF(s2));
        }
        if (base - NB < NB) {   // a head row of panel Bp+1: take row r - Sb
          const int64_t r2 = r - Sb;
          row[u] = r2;
#pragma unroll
          for (int c = 0; c < NC; ++c) {
            v[u][c] = nxt[u][c];
            const int64_t rn = r2 - Sb;
            nxt[u][c] = (rn >= 0 && rn < n && c < ncol) ? Yo[(int64_t)(c0 + c) * a.ldy + rn] : zero;
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(EMPTY(s));
    }
  }
}

template <typename CT, int NC, int SPT, int REGS>
__global__ void __maxnreg__(REGS) band_solve_la_kernel(SolveArgsT<CT> a) {
  la_cta<CT, NC, SPT>(a, blockIdx.y, blockIdx.x);
}

// The look-ahead solve of many independent problems in one launch, laid out as
// band_solve_batch_kernel: CTA b serves solve cta[b].x, pole cta[b].y, column group cta[b].z;
// the block size is that of the widest band (a narrower solve leaves the extra update slots
// idle) and each solve has its own staged-panel count.
template <typename CT, int NC, int SPT, int REGS>
__global__ void __maxnreg__(REGS) band_solve_la_batch_kernel(const SolveArgsT<CT>* items,
                                                             const int4* cta) {
  const int4 m = cta[blockIdx.x];
  const SolveArgsT<CT> a = items[m.x];
  la_cta<CT, NC, SPT>(a, m.y, m.z);
}

// ----------------------------------------------------------------------------------------------
// Block transforms, computed once per factorisation (one warp per (panel, pole)):
//  forward: the set H of a panel's NB steps (head rows j0..j0+NB-1, then for step jj its pivot
//    row if it lies below the head and no earlier step named it; -1 = absent) and the 16x16
//    matrix T such that the panel's interleaved swaps and eliminations restricted to H are
//    H <- T H (T[:, m] = the steps applied to the unit vector of member m), stored by columns
//    (T[i][m] at m*16 + i, so that the 16 outputs of one member read 16 consecutive words);
//  backward: inv(U_block), the 8x8 inverse of U's diagonal block of the panel (rows and
//    columns >= n are zero).
// T and inv(U_block) are written in complex128 and, when T32/Ui32 are given, complex64.
__device__ __forceinline__ cplx ld_c(const cplx* p) { return *p; }
__device__ __forceinline__ cplx ld_c(const float2* p) {
  const float2 v = *p;
  return make_double2(v.x, v.y);
}

// AT: element type of the band factors and 1/u_jj (complex128, or complex64 from the FP32 LU;
// the transforms are then formed in FP64 from the complex64 entries and rounded).
template <typename AT>
__global__ void block_transform_kernel(int64_t n, int64_t n_pad, int kl, int ldab, const AT* AB,
                                       const int* piv, const AT* dinv, cplx* Tout, int* Hout,
                                       cplx* Uiout, float2* T32, float2* Ui32) {
  const int P = blockIdx.x, pole = blockIdx.y, lane = threadIdx.x;
  const int kv = 2 * kl;
  const int64_t npan = n_pad / NB;
  const int64_t j0 = (int64_t)P * NB;
  const int nvalid = (int)((n - j0) < NB ? (n - j0) : NB);
  const AT* A = AB + (int64_t)pole * n_pad * ldab;
  const int* pv = piv + (int64_t)pole * n_pad;
  const AT* di = dinv + (int64_t)pole * n_pad;
  int64_t pst[NB];
#pragma unroll
  for (int jj = 0; jj < NB; ++jj) pst[jj] = (jj < nvalid) ? pv[j0 + jj] : -1;
  auto hidx = [&](int64_t r) -> int {
    if (r >= j0 && r < j0 + NB) return (int)(r - j0);
    for (int jj = 0; jj < nvalid; ++jj)
      if (pst[jj] == r) return NB + jj;
    return -1;
  };
  auto hrow = [&](int l) -> int64_t {
    if (l < NB) return j0 + l;
    if (l < 2 * NB) {
      const int jj = l - NB;
      if (jj < nvalid && pst[jj] >= j0 + NB && hidx(pst[jj]) == l) return pst[jj];
    }
    return -1;
  };
  const int64_t myrow = hrow(lane);
  const int64_t base = (int64_t)pole * npan + P;
  if (lane < 16) Hout[base * 16 + lane] = (int)myrow;
  for (int m = 0; m < 16; ++m) {
    const bool present = hrow(m) >= 0;
    cplx val = make_double2((lane == m && present) ? 1.0 : 0.0, 0.0);
    if (present) {
      for (int jj = 0; jj < nvalid; ++jj) {
        const int64_t j = j0 + jj;
        const int b = hidx(pst[jj]);
        const cplx x = make_double2(__shfl_sync(0xffffffffu, val.x, b), __shfl_sync(0xffffffffu, val.y, b));
        const cplx va = make_double2(__shfl_sync(0xffffffffu, val.x, jj),
                                     __shfl_sync(0xffffffffu, val.y, jj));
        if (lane == jj) val = x;
        else if (lane == b) val = va;
        if (myrow > j && myrow <= j + kl) val = cfms(ld_c(A + j * ldab + kv + (myrow - j)), x, val);
      }
    }
    if (lane < 16) {
      const cplx t = (myrow >= 0 && present) ? val : make_double2(0, 0);
      if (Tout) Tout[base * 256 + m * 16 + lane] = t;
      if (T32) T32[base * 256 + m * 16 + lane] = make_float2((float)t.x, (float)t.y);
    }
  }
  // column b of inv(U_block) by back substitution: U(r, c) = A[c*ldab + kv + r - c], r <= c
  if (lane < NB) {
    const int b = lane;
    cplx z[NB];
#pragma unroll
    for (int i = 0; i < NB; ++i) z[i] = make_double2(0, 0);
    for (int i = b; i >= 0; --i) {
      const int64_t r = j0 + i;
      cplx acc = make_double2(i == b ? 1.0 : 0.0, 0.0);
      for (int c = i + 1; c <= b; ++c)
        if (c - i <= kv && j0 + c < n) acc = cfms(ld_c(A + (j0 + c) * ldab + kv + (r - (j0 + c))), z[c], acc);
      z[i] = (r < n) ? cmul(acc, ld_c(di + r)) : make_double2(0, 0);
    }
    for (int i = 0; i < NB; ++i) {
      const cplx t = z[i];
      if (Uiout) Uiout[base * 64 + i * NB + b] = t;
      if (Ui32) Ui32[base * 64 + i * NB + b] = make_float2((float)t.x, (float)t.y);
    }
  }
}

void launch_block_transforms(int q, int64_t n, int64_t n_pad, int kl, int ldab, const cplx* AB,
                             const int* piv, const cplx* dinv, cplx* T, int* H, cplx* Ui,
                             float2* T32, float2* Ui32, cudaStream_t s) {
  dim3 grid((unsigned)(n_pad / NB), (unsigned)q);
  block_transform_kernel<cplx><<<grid, 32, 0, s>>>(n, n_pad, kl, ldab, AB, piv, dinv, T, H, Ui, T32, Ui32); ie_count_launch();
}

void launch_block_transforms(int q, int64_t n, int64_t n_pad, int kl, int ldab, const float2* AB,
                             const int* piv, const float2* dinv, int* H, float2* T32,
                             float2* Ui32, cudaStream_t s) {
  dim3 grid((unsigned)(n_pad / NB), (unsigned)q);
  block_transform_kernel<float2><<<grid, 32, 0, s>>>(n, n_pad, kl, ldab, AB, piv, dinv, nullptr, H, nullptr, T32, Ui32); ie_count_launch();
}

template <typename CT, int NC, int SPT, int REGS>
static cudaError_t launch_solve_r(const SolveArgsT<CT>& a, int q, int threads, size_t smem,
                                  cudaStream_t s) {
  auto kfn = band_solve_kernel<CT, NC, SPT, REGS>;
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

template <typename CT, int NC, int SPT>
static cudaError_t launch_solve_t(const SolveArgsT<CT>& a, int q, int threads, size_t smem,
                                  cudaStream_t s) {
  if (threads <= 16 * 32) return launch_solve_r<CT, NC, SPT, 112>(a, q, threads, smem, s);
  return launch_solve_r<CT, NC, SPT, 96>(a, q, threads, smem, s);
}

template <typename CT, int NC, int SPT, int REGS>
static cudaError_t launch_pipe_r(const SolveArgsT<CT>& a, int q, int threads, size_t smem,
                                 cudaStream_t s) {
  auto kfn = band_solve_pipe_kernel<CT, NC, SPT, REGS>;
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

// register budget by warps per sub-partition: ceil(W/4) * 32 * REGS <= 16384
template <typename CT, int NC, int SPT>
static cudaError_t launch_pipe_t(const SolveArgsT<CT>& a, int q, int threads, size_t smem,
                                 cudaStream_t s) {
  const int wps = (threads / 32 + 3) / 4;
  if (wps <= 4) return launch_pipe_r<CT, NC, SPT, 128>(a, q, threads, smem, s);
  if (wps <= 5) return launch_pipe_r<CT, NC, SPT, 96>(a, q, threads, smem, s);
  return cudaErrorInvalidValue;
}

template <typename CT, int NC, int SPT, int REGS>
static cudaError_t launch_la_r(const SolveArgsT<CT>& a, int q, int threads, size_t smem,
                               cudaStream_t s) {
  auto kfn = band_solve_la_kernel<CT, NC, SPT, REGS>;
  cudaError_t e = ie_smem_optin((const void*)kfn);
  if (e != cudaSuccess) return e;
  int blocks = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kfn, threads, smem);
  if (e != cudaSuccess) return e;
  if (blocks < 1) return cudaErrorLaunchOutOfResources;
  dim3 grid((unsigned)((a.k + NC - 1) / NC), (unsigned)q);
  kfn<<<grid, threads, smem, s>>>(a); ie_count_launch();
  return cudaGetLastError();
}

template <typename CT, int NC, int SPT>
static cudaError_t launch_la_t(const SolveArgsT<CT>& a, int q, int threads, size_t smem,
                               cudaStream_t s) {
  const int wps = (threads / 32 + 3) / 4;
  if (wps <= 3) return launch_la_r<CT, NC, SPT, 168>(a, q, threads, smem, s);
  if (wps <= 4) return launch_la_r<CT, NC, SPT, 128>(a, q, threads, smem, s);
  if (wps <= 5) return launch_la_r<CT, NC, SPT, 96>(a, q, threads, smem, s);
  return cudaErrorInvalidValue;
}

// One launch shape: NC right-hand sides per CTA, SPT window slots per thread, at most
// `stages` staged panels; pipe = 1 for the warp-specialised kernel, 2 for its look-ahead form.
struct SolveCfg {
  int nc, spt, stages, pipe;
};

// threads, stages and dynamic shared memory of a shape; false if the shape cannot hold the band
template <typename CT>
static bool shape_for(SolveArgsT<CT>& a, const SolveCfg& c, int* threads, size_t* smem) {
  const int slots = a.kv > NB ? a.kv : NB;     // backward window (at least the forward's)
  if (c.pipe == 2) {
    // update warps for the window (at least two heads deep), the head warps (two right-hand
    // sides each) and the producer warp
    const int slots2 = a.kv > 2 * NB ? a.kv : 2 * NB;
    const int nh = c.nc >= 2 ? c.nc / 2 : 1;
    const int wu = ((slots2 + c.spt - 1) / c.spt + 31) / 32;
    *threads = (wu + nh + 1) * 32;
    if (*threads > 640) return false;
    const size_t fwdb = (size_t)NB * a.klp * sizeof(CT) + 256 * sizeof(CT) + 32 * sizeof(int);
    const size_t bwdb = (size_t)NB * a.kvp * sizeof(CT) + 64 * sizeof(CT);
    const size_t fac = ((fwdb > bwdb ? fwdb : bwdb) + 127) & ~(size_t)127;
    const size_t stage_bytes = (fac + 2 * (size_t)16 * c.nc * sizeof(CT) + 127) & ~(size_t)127;
    const size_t budget = 210 * 1024;
    int nstage = c.stages > 3 ? c.stages : 3;
    auto need = [&](int k) { return ((4 * (size_t)k * 8 + 127) & ~(size_t)127) + k * stage_bytes; };
    while (nstage > 3 && need(nstage) > budget) --nstage;
    if (need(nstage) > budget) return false;
    a.nstage = nstage;
    *smem = need(nstage);
    return true;
  }
  if (c.pipe) {
    // update warps for the window, then the head warp and the producer warp
    const int wu = ((slots + c.spt - 1) / c.spt + 31) / 32;
    *threads = (wu + 2) * 32;
    if (*threads > 640) return false;
    const size_t fwdb = (size_t)NB * a.klp * sizeof(CT) + 256 * sizeof(CT) + 16 * sizeof(int);
    const size_t bwdb = (size_t)NB * a.kvp * sizeof(CT) + 64 * sizeof(CT);
    const size_t fac = ((fwdb > bwdb ? fwdb : bwdb) + 127) & ~(size_t)127;
    const size_t stage_bytes = (fac + 2 * (size_t)16 * c.nc * sizeof(CT) + 127) & ~(size_t)127;
    const size_t budget = 200 * 1024;
    // a power of two (the kernel indexes the ring by masks): 4 stages when they fit, else 2
    int nstage = c.stages >= 4 ? 4 : 2;
    if (((4 * (size_t)nstage * 8 + 127) & ~(size_t)127) + nstage * stage_bytes > budget) nstage = 2;
    const size_t need = ((4 * (size_t)nstage * 8 + 127) & ~(size_t)127) + nstage * stage_bytes;
    if (need > budget) return false;
    a.nstage = nstage;
    *smem = need;
    return true;
  }
  if ((slots + c.spt - 1) / c.spt > 576) return false;
  *threads = ((slots + c.spt - 1) / c.spt + 31) / 32 * 32;
  const size_t fwdb = (size_t)NB * a.klp * sizeof(CT) + 256 * sizeof(CT) + 16 * sizeof(int);
  const size_t bwdb = (size_t)NB * a.kvp * sizeof(CT) + 64 * sizeof(CT);
  const size_t stage_bytes = ((fwdb > bwdb ? fwdb : bwdb) + 127) & ~(size_t)127;
  // mbarriers, then hd and xs [NB][NC], hv and hv2 [16][NC], partials [NPART][16][NC],
  // alignment slack
  const size_t fixed = 128 + (size_t)(2 * NB + 32 + NPART * 16) * c.nc * sizeof(CT) + 256;
  const size_t budget = 200 * 1024;
  if (fixed + 2 * stage_bytes > budget) return false;
  int nstage = (int)((budget - fixed) / stage_bytes);
  if (nstage > c.stages) nstage = c.stages;
  a.nstage = nstage;
  *smem = fixed + (size_t)nstage * stage_bytes;
  return true;
}

template <typename CT>
static cudaError_t launch_cfg(SolveArgsT<CT> a, int q, const SolveCfg& c, cudaStream_t s) {
  int threads;
  size_t smem;
  if (!shape_for(a, c, &threads, &smem)) return cudaErrorInvalidValue;
#define IE_SOLVE_CASE(NC_, SPT_)                                                             \
  if (c.nc == NC_ && c.spt == SPT_)                                                          \
    return c.pipe == 2 ? launch_la_t<CT, NC_, SPT_>(a, q, threads, smem, s)                  \
           : c.pipe    ? launch_pipe_t<CT, NC_, SPT_>(a, q, threads, smem, s)                \
                       : launch_solve_t<CT, NC_, SPT_>(a, q, threads, smem, s);
  IE_SOLVE_CASE(1, 1) IE_SOLVE_CASE(2, 1) IE_SOLVE_CASE(4, 1)
  IE_SOLVE_CASE(1, 2) IE_SOLVE_CASE(2, 2) IE_SOLVE_CASE(4, 2)
  if constexpr (sizeof(CT) == sizeof(float2)) {
    IE_SOLVE_CASE(8, 1) IE_SOLVE_CASE(8, 2)
  }
#undef IE_SOLVE_CASE
  return cudaErrorInvalidValue;
}

static int pick_nc(int q, int k, int sms, int ncmax) {
  // the smallest NC that keeps q * ceil(k/NC) CTAs within one wave
  for (int c = 1; c <= ncmax; c *= 2)
    if ((int64_t)q * ((k + c - 1) / c) <= sms) return c;
  return ncmax;
}

// Online autotuner of the launch shape. For each (element type, band, poles, block width
// rounded up to a power of two) the first launches each use a different candidate shape,
// timed with CUDA events; once all are timed, the fastest is used. Every candidate does the
// same arithmetic per column (results are identical), so tuning costs no extra work.
// IE_SOLVE_TUNE=0 in the environment disables it (the default shape is used).
namespace {
struct TuneKey {
  int esize, kl, q, kb;
  bool operator<(const TuneKey& o) const {
    return std::tie(esize, kl, q, kb) < std::tie(o.esize, o.kl, o.q, o.kb);
  }
};
struct TuneState {
  std::vector<SolveCfg> cand;
  std::vector<cudaEvent_t> e0, e1;
  std::vector<float> ms;   // < 0: pending; +inf: shape not launchable
  int next = 0, best = -1;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneState> g_tune;
bool tune_enabled() {
  static const bool on = [] {
    const char* e = getenv("IE_SOLVE_TUNE");
    return !(e && e[0] == '0');
  }();
  return on;
}
// IE_SOLVE_TUNE_LOG=1: print each tuning decision (candidate shapes and times) to stderr
bool tune_log() {
  static const bool on = [] {
    const char* e = getenv("IE_SOLVE_TUNE_LOG");
    return e && e[0] == '1';
  }();
  return on;
}
}  // namespace

namespace {
std::atomic<int> g_last_kernel[2] = {-1, -1};
}  // namespace
int band_solve_last_kernel(int fp32) { return g_last_kernel[fp32 ? 1 : 0].load(); }

template <typename CT>
static cudaError_t launch_tuned(const SolveArgsT<CT>& a, int q, cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const bool fp32 = sizeof(CT) == sizeof(float2);
  const int spt0 = ((a.kv > NB ? a.kv : NB) > 576) ? 2 : 1;
  const SolveCfg dflt{pick_nc(q, a.k, sms, fp32 ? 8 : 4), spt0, 6, 0};
  if (!tune_enabled()) {
    g_last_kernel[fp32 ? 1 : 0] = dflt.pipe;
    return launch_cfg(a, q, dflt, s);
  }
  int kb = 1;
  while (kb < a.k) kb *= 2;
  const TuneKey key{(int)sizeof(CT), a.kl, q, kb};
  SolveCfg use = dflt;
  int slot = -1;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneState& T = g_tune[key];
    if (T.cand.empty()) {
      std::vector<SolveCfg> c = {dflt, {2, 2, 3, 0}, {4, 2, 3, 0}, {2, 1, 3, 0}, {1, 2, 3, 0},
                                 {4, 1, 3, 0}};
      if (fp32) {
        c.push_back({8, 1, 3, 0});
        c.push_back({8, 2, 2, 0});
        c.push_back({2, 2, 2, 0});
      }
      // the warp-specialised kernel
      c.push_back({dflt.nc, spt0, 4, 1});
      c.push_back({2, spt0, 4, 1});
      c.push_back({4, 2, 4, 1});
      c.push_back({2, 2, 4, 1});
      if (fp32) {
        c.push_back({8, spt0, 4, 1});
        c.push_back({8, 2, 3, 1});
      }
      // its look-ahead form (as many stages as fit, at least three; the second shape with
      // exactly three)
      c.push_back({4, spt0, 6, 2});
      c.push_back({4, 2, 6, 2});
      c.push_back({4, 2, 3, 2});
      c.push_back({2, spt0, 6, 2});
      c.push_back({2, 2, 6, 2});
      if (fp32) {
        c.push_back({8, spt0, 6, 2});
        c.push_back({8, 2, 6, 2});
      }
      for (const SolveCfg& x : c) {
        if (x.spt < spt0) continue;
        bool dup = false;
        for (const SolveCfg& y : T.cand)
          dup |= (y.nc == x.nc && y.spt == x.spt && y.stages == x.stages && y.pipe == x.pipe);
        if (!dup) T.cand.push_back(x);
      }
      T.e0.resize(T.cand.size());
      T.e1.resize(T.cand.size());
      for (size_t i = 0; i < T.cand.size(); ++i) {
        cudaEventCreate(&T.e0[i]);
        cudaEventCreate(&T.e1[i]);
      }
      T.ms.assign(T.cand.size(), -1.0f);
    }
    if (T.best >= 0) {
      use = T.cand[T.best];
    } else {
      bool all = T.next == (int)T.cand.size();
      for (int i = 0; i < T.next; ++i) {
        if (T.ms[i] >= 0.0f) continue;
        if (cudaEventQuery(T.e1[i]) == cudaSuccess) cudaEventElapsedTime(&T.ms[i], T.e0[i], T.e1[i]);
        else { cudaGetLastError(); all = false; }
      }
      if (all) {
        int b = 0;
        for (int i = 1; i < (int)T.cand.size(); ++i)
          if (T.ms[i] < T.ms[b]) b = i;
        T.best = b;
        use = T.cand[b];
        if (tune_log()) {
          fprintf(stderr, "band solve tuner (elem %d B, kl %d, q %d, k <= %d):", key.esize, key.kl,
                  key.q, key.kb);
          for (size_t i = 0; i < T.cand.size(); ++i)
            fprintf(stderr, " [%s nc %d spt %d stages %d: %.3f ms]",
                    T.cand[i].pipe == 2 ? "look-ahead" : T.cand[i].pipe ? "pipe" : "sync",
                    T.cand[i].nc, T.cand[i].spt, T.cand[i].stages, T.ms[i]);
          fprintf(stderr, " -> %d\n", b);
        }
      } else if (T.next < (int)T.cand.size()) {
        slot = T.next++;
        use = T.cand[slot];
      }
    }
    if (slot >= 0) cudaEventRecord(T.e0[slot], s);
  }
  cudaError_t e = launch_cfg(a, q, use, s);
  g_last_kernel[fp32 ? 1 : 0] = e == cudaSuccess ? use.pipe : dflt.pipe;
  if (slot >= 0) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneState& T = g_tune[key];
    if (e == cudaSuccess) {
      cudaEventRecord(T.e1[slot], s);
    } else {   // shape not launchable here: never pick it, compute this call with the default
      cudaGetLastError();
      T.ms[slot] = 3.0e38f;
      cudaEventRecord(T.e1[slot], s);
      e = launch_cfg(a, q, dflt, s);
    }
  }
  return e;
}

cudaError_t launch_band_solve(int q, int64_t n, int kl, int64_t n_pad, const cplx* L64,
                              const cplx* U64, const int* piv, const cplx* dinv, const cplx* Tb, const int* Hb,
                              const cplx* Ub, const cplx* d_weights, const cplx* RHS, int64_t ldr,
                              int k, cplx* Xp, int64_t ldx, int64_t xstride, int* status,
                              cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  SolveArgsT<cplx> a{};
  a.n = n; a.n_pad = n_pad; a.kl = kl; a.kv = 2 * kl; a.klp = kl; a.kvp = 2 * kl; a.k = k;
  a.mode = 0;
  a.L = L64; a.U = U64; a.ldl = kl; a.ldu = 2 * kl;
  a.lstride = n_pad * kl; a.ustride = n_pad * 2 * kl;
  a.piv = piv; a.dinv = dinv; a.weights = d_weights;
  a.Tb = Tb; a.Hb = Hb; a.Ub = Ub;
  a.RHS = RHS; a.ldr = ldr; a.rstride = 0;
  a.Y = Xp; a.ldy = ldx; a.ystride = xstride;
  a.X = Xp; a.ldx = ldx; a.xstride = xstride;
  a.status = status;
  return launch_tuned(a, q, s);
}

cudaError_t launch_band_solve32(int q, int64_t n, int kl, int64_t n_pad, const float2* L32,
                                int64_t ldl, const float2* U32, int64_t ldu, const int* piv,
                                const float2* dinv32, const float2* T32, const int* Hb,
                                const float2* Ui32, const cplx* d_weights, const float2* RHS,
                                int64_t ldr, int64_t rstride, int k, float2* Y32, int64_t ldy,
                                int64_t ystride, cplx* X, int64_t ldx, int64_t xstride,
                                int accumulate, int* status, cudaStream_t s) {
  if (k <= 0) return cudaSuccess;
  SolveArgsT<float2> a{};
  a.n = n; a.n_pad = n_pad; a.kl = kl; a.kv = 2 * kl;
  a.klp = (int)ldl; a.kvp = (int)ldu;   // padded column lengths = column strides
  a.k = k; a.mode = accumulate ? 3 : 1;
  a.L = L32; a.U = U32; a.ldl = ldl; a.ldu = ldu;
  a.lstride = n_pad * ldl; a.ustride = n_pad * ldu;
  a.piv = piv; a.dinv = dinv32; a.weights = d_weights;
  a.Tb = T32; a.Hb = Hb; a.Ub = Ui32;
  a.RHS = RHS; a.ldr = ldr; a.rstride = rstride;
  a.Y = Y32; a.ldy = ldy; a.ystride = ystride;
  a.X = X; a.ldx = ldx; a.xstride = xstride;
  a.status = status;
  return launch_tuned(a, q, s);
}

// ----------------------------------------------------------------------------------------------
// Batched band solves: the solves of many problems in one launch per element type
// (band_solve_batch_kernel). Each added solve is described exactly as launch_band_solve /
// launch_band_solve32 would launch it; the launch uses one shape for all of them (NC = 4 right-
// hand sides per CTA, the block size of the widest band) and gives each solve the staged panels
// that fit the common shared-memory size. CTAs are ordered by decreasing work so the longest
// solves start first.
struct BandSolveBatch {
  std::vector<SolveArgsT<cplx>> a64;
  std::vector<int> q64;
  std::vector<SolveArgsT<float2>> a32;
  std::vector<int> q32;
  void* d_items = nullptr;
  size_t items_cap = 0;
  int4* d_cta = nullptr;
  size_t cta_cap = 0;
  std::vector<int4> cta;
};

BandSolveBatch* band_solve_batch_create() { return new BandSolveBatch(); }
void band_solve_batch_destroy(BandSolveBatch* b) {
  if (!b) return;
  cudaFree(b->d_items);
  cudaFree(b->d_cta);
  delete b;
}
void band_solve_batch_clear(BandSolveBatch* b) {
  b->a64.clear();
  b->q64.clear();
  b->a32.clear();
  b->q32.clear();
}
int band_solve_batch_size(const BandSolveBatch* b) { return (int)(b->a64.size() + b->a32.size()); }

void band_solve_batch_add64(BandSolveBatch* b, int q, int64_t n, int kl, int64_t n_pad,
                            const cplx* L64, const cplx* U64, const int* piv, const cplx* dinv,
                            const cplx* Tb, const int* Hb, const cplx* Ub, const cplx* d_weights,
                            const cplx* RHS, int64_t ldr, int k, cplx* Xp, int64_t ldx,
                            int64_t xstride, int* status) {
  if (k <= 0) return;
  SolveArgsT<cplx> a{};
  a.n = n; a.n_pad = n_pad; a.kl = kl; a.kv = 2 * kl; a.klp = kl; a.kvp = 2 * kl; a.k = k;
  a.mode = 0;
  a.L = L64; a.U = U64; a.ldl = kl; a.ldu = 2 * kl;
  a.lstride = n_pad * kl; a.ustride = n_pad * 2 * kl;
  a.piv = piv; a.dinv = dinv; a.weights = d_weights;
  a.Tb = Tb; a.Hb = Hb; a.Ub = Ub;
  a.RHS = RHS; a.ldr = ldr; a.rstride = 0;
  a.Y = Xp; a.ldy = ldx; a.ystride = xstride;
  a.X = Xp; a.ldx = ldx; a.xstride = xstride;
  a.status = status;
  b->a64.push_back(a);
  b->q64.push_back(q);
}

void band_solve_batch_add32(BandSolveBatch* b, int q, int64_t n, int kl, int64_t n_pad,
                            const float2* L32, int64_t ldl, const float2* U32, int64_t ldu,
                            const int* piv, const float2* dinv32, const float2* T32,
                            const int* Hb, const float2* Ui32, const cplx* d_weights,
                            const float2* RHS, int64_t ldr, int64_t rstride, int k, float2* Y32,
                            int64_t ldy, int64_t ystride, cplx* X, int64_t ldx, int64_t xstride,
                            int accumulate, int* status) {
  if (k <= 0) return;
  SolveArgsT<float2> a{};
  a.n = n; a.n_pad = n_pad; a.kl = kl; a.kv = 2 * kl;
  a.klp = (int)ldl; a.kvp = (int)ldu;
  a.k = k; a.mode = accumulate ? 3 : 1;
  a.L = L32; a.U = U32; a.ldl = ldl; a.ldu = ldu;
  a.lstride = n_pad * ldl; a.ustride = n_pad * ldu;
  a.piv = piv; a.dinv = dinv32; a.weights = d_weights;
  a.Tb = T32; a.Hb = Hb; a.Ub = Ui32;
  a.RHS = RHS; a.ldr = ldr; a.rstride = rstride;
  a.Y = Y32; a.ldy = ldy; a.ystride = ystride;
  a.X = X; a.ldx = ldx; a.xstride = xstride;
  a.status = status;
  b->a32.push_back(a);
  b->q32.push_back(q);
}

template <typename CT, int SPT, int REGS>
static cudaError_t batch_launch_r(BandSolveBatch* b, std::vector<SolveArgsT<CT>>& items,
                                  int threads, size_t smem, cudaStream_t s) {
  auto kfn = band_solve_batch_kernel<CT, 4, SPT, REGS>;
  cudaError_t e = ie_smem_optin((const void*)kfn);
  if (e != cudaSuccess) return e;
  int blocks = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kfn, threads, smem);
  if (e != cudaSuccess) return e;
  if (blocks < 1) return cudaErrorLaunchOutOfResources;
  const size_t ib = items.size() * sizeof(SolveArgsT<CT>);
  if (ib > b->items_cap) {
    cudaFree(b->d_items);
    b->d_items = nullptr;
    e = cudaMalloc(&b->d_items, ib);
    if (e != cudaSuccess) { b->items_cap = 0; return e; }
    b->items_cap = ib;
  }
  if (b->cta.size() > b->cta_cap) {
    cudaFree(b->d_cta);
    b->d_cta = nullptr;
    e = cudaMalloc(&b->d_cta, b->cta.size() * sizeof(int4));
    if (e != cudaSuccess) { b->cta_cap = 0; return e; }
    b->cta_cap = b->cta.size();
  }
  // pageable sources: the copies complete before cudaMemcpyAsync returns to the host
  e = cudaMemcpyAsync(b->d_items, items.data(), ib, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(b->d_cta, b->cta.data(), b->cta.size() * sizeof(int4),
                      cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  kfn<<<(unsigned)b->cta.size(), threads, smem, s>>>((const SolveArgsT<CT>*)b->d_items, b->d_cta);
  ie_count_launch();
  return cudaGetLastError();
}

template <typename CT, int SPT, int REGS>
static cudaError_t batch_la_launch_r(BandSolveBatch* b, std::vector<SolveArgsT<CT>>& items,
                                     int threads, size_t smem, cudaStream_t s) {
  auto kfn = band_solve_la_batch_kernel<CT, 4, SPT, REGS>;
  cudaError_t e = ie_smem_optin((const void*)kfn);
  if (e != cudaSuccess) return e;
  int blocks = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kfn, threads, smem);
  if (e != cudaSuccess) return e;
  if (blocks < 1) return cudaErrorLaunchOutOfResources;
  const size_t ib = items.size() * sizeof(SolveArgsT<CT>);
  if (ib > b->items_cap) {
    cudaFree(b->d_items);
    b->d_items = nullptr;
    e = cudaMalloc(&b->d_items, ib);
    if (e != cudaSuccess) { b->items_cap = 0; return e; }
    b->items_cap = ib;
  }
  if (b->cta.size() > b->cta_cap) {
    cudaFree(b->d_cta);
    b->d_cta = nullptr;
    e = cudaMalloc(&b->d_cta, b->cta.size() * sizeof(int4));
    if (e != cudaSuccess) { b->cta_cap = 0; return e; }
    b->cta_cap = b->cta.size();
  }
  // pageable sources: the copies complete before cudaMemcpyAsync returns to the host
  e = cudaMemcpyAsync(b->d_items, items.data(), ib, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(b->d_cta, b->cta.data(), b->cta.size() * sizeof(int4),
                      cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  kfn<<<(unsigned)b->cta.size(), threads, smem, s>>>((const SolveArgsT<CT>*)b->d_items, b->d_cta);
  ie_count_launch();
  return cudaGetLastError();
}

// The batch as one look-ahead launch (4 right-hand sides per CTA, two window slots per thread
// above 256 slots): each solve gets the staged panels that fit the common shared-memory size,
// at least three. Returns cudaErrorInvalidValue when some solve does not fit (the caller then
// uses the synchronised batch kernel).
template <typename CT>
static cudaError_t batch_la_launch_t(BandSolveBatch* b, std::vector<SolveArgsT<CT>>& items,
                                     const std::vector<int>& qs, cudaStream_t s) {
  constexpr int NCB = 4, NHB = 2;
  int slots = 2 * NB;
  for (auto& a : items) slots = std::max(slots, a.kv);
  const int spt = slots > 256 ? 2 : 1;
  const int wu = ((slots + spt - 1) / spt + 31) / 32;
  const int threads = (wu + NHB + 1) * 32;
  if (threads > 640) return cudaErrorInvalidValue;
  const size_t budget = 210 * 1024;
  auto stage_of = [&](const SolveArgsT<CT>& a) {
    const size_t fwdb = (size_t)NB * a.klp * sizeof(CT) + 256 * sizeof(CT) + 32 * sizeof(int);
    const size_t bwdb = (size_t)NB * a.kvp * sizeof(CT) + 64 * sizeof(CT);
    const size_t fac = ((fwdb > bwdb ? fwdb : bwdb) + 127) & ~(size_t)127;
    return (fac + 2 * (size_t)16 * NCB * sizeof(CT) + 127) & ~(size_t)127;
  };
  auto need = [&](int k, size_t st) { return ((4 * (size_t)k * 8 + 127) & ~(size_t)127) + k * st; };
  size_t smem = 0;
  for (auto& a : items) {
    const size_t st = stage_of(a);
    if (need(3, st) > budget) return cudaErrorInvalidValue;
    int ns = 3;
    while (ns < 6 && need(ns + 1, st) <= budget) ++ns;
    a.nstage = ns;
    smem = std::max(smem, need(ns, st));
  }
  std::vector<int> ord(items.size());
  for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
    return items[x].n * (items[x].kl + items[x].kv) > items[y].n * (items[y].kl + items[y].kv);
  });
  b->cta.clear();
  for (int i : ord)
    for (int p = 0; p < qs[i]; ++p)
      for (int g = 0; g * NCB < items[i].k; ++g) b->cta.push_back(make_int4(i, p, g, 0));
  const int wps = (threads / 32 + 3) / 4;
  if (spt == 1) {
    if (wps <= 3) return batch_la_launch_r<CT, 1, 168>(b, items, threads, smem, s);
    if (wps <= 4) return batch_la_launch_r<CT, 1, 128>(b, items, threads, smem, s);
    if (wps <= 5) return batch_la_launch_r<CT, 1, 96>(b, items, threads, smem, s);
    return cudaErrorInvalidValue;
  }
  if (wps <= 3) return batch_la_launch_r<CT, 2, 168>(b, items, threads, smem, s);
  if (wps <= 4) return batch_la_launch_r<CT, 2, 128>(b, items, threads, smem, s);
  if (wps <= 5) return batch_la_launch_r<CT, 2, 96>(b, items, threads, smem, s);
  return cudaErrorInvalidValue;
}

template <typename CT>
static cudaError_t batch_launch_t(BandSolveBatch* b, std::vector<SolveArgsT<CT>>& items,
                                  const std::vector<int>& qs, cudaStream_t s) {
  if (items.empty()) return cudaSuccess;
  // the look-ahead kernel when every solve fits it (IE_BATCH_SYNC=1: always the synchronised one)
  static const bool force_sync = [] {
    const char* e = getenv("IE_BATCH_SYNC");
    return e && e[0] == '1';
  }();
  if (!force_sync) {
    std::vector<SolveArgsT<CT>> la = items;
    const cudaError_t e = batch_la_launch_t(b, la, qs, s);
    if (e != cudaErrorInvalidValue) return e;
  }
  constexpr int NCB = 4;
  int slots = NB;
  for (auto& a : items) slots = std::max(slots, a.kv);
  const int spt = slots > 576 ? 2 : 1;
  if ((slots + spt - 1) / spt > 576) return cudaErrorInvalidValue;
  const int threads = ((slots + spt - 1) / spt + 31) / 32 * 32;
  const size_t fixed = 128 + (size_t)(2 * NB + 32 + NPART * 16) * NCB * sizeof(CT) + 256;
  const size_t budget = 200 * 1024;
  size_t smem = 0;
  for (auto& a : items) {
    const size_t fwdb = (size_t)NB * a.klp * sizeof(CT) + 256 * sizeof(CT) + 16 * sizeof(int);
    const size_t bwdb = (size_t)NB * a.kvp * sizeof(CT) + 64 * sizeof(CT);
    const size_t st = ((fwdb > bwdb ? fwdb : bwdb) + 127) & ~(size_t)127;
    if (fixed + 2 * st > budget) return cudaErrorInvalidValue;
    int ns = (int)((budget - fixed) / st);
    if (ns > 6) ns = 6;
    a.nstage = ns;
    smem = std::max(smem, fixed + (size_t)ns * st);
  }
  // CTAs, longest solves first (work ~ n * (kl + kv) per CTA)
  std::vector<int> ord(items.size());
  for (size_t i = 0; i < ord.size(); ++i) ord[i] = (int)i;
  std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
    return items[x].n * (items[x].kl + items[x].kv) > items[y].n * (items[y].kl + items[y].kv);
  });
  b->cta.clear();
  for (int i : ord)
    for (int p = 0; p < qs[i]; ++p)
      for (int g = 0; g * NCB < items[i].k; ++g) b->cta.push_back(make_int4(i, p, g, 0));
  if (spt == 1) {
    if (threads <= 16 * 32) return batch_launch_r<CT, 1, 112>(b, items, threads, smem, s);
    return batch_launch_r<CT, 1, 96>(b, items, threads, smem, s);
  }
  if (threads <= 16 * 32) return batch_launch_r<CT, 2, 112>(b, items, threads, smem, s);
  return batch_launch_r<CT, 2, 96>(b, items, threads, smem, s);
}

cudaError_t band_solve_batch_launch(BandSolveBatch* b, cudaStream_t s) {
  cudaError_t e = batch_launch_t(b, b->a64, b->q64, s);
  if (e != cudaSuccess) return e;
  return batch_launch_t(b, b->a32, b->q32, s);
}

// C ABI of the interior eigensolver (include/ie.h): handle life cycle, the composite-rule
// coefficients (Eq. pwtp; Thm 2), the filter (Alg. 1), HSRR (extraction steps of Alg.
// SIsketch) and the two drivers (Alg. 1, Alg. 2). Host code orchestrates kernels on one stream;
// the GMRES loop reads k residuals back per Arnoldi step for its convergence test.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <complex>
#include <cstring>
#include <limits>
#include <atomic>
#include <numeric>
#include <set>
#include <thread>
#include <vector>

#include "ie_internal.cuh"

typedef std::complex<double> zc;

namespace {
inline cplx to_c(zc z) { return make_double2(z.real(), z.imag()); }
inline zc to_z(cplx c) { return zc(c.x, c.y); }
inline zc to_z(ie_complex c) { return zc(c.re, c.im); }

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

ie_status map_err(cudaError_t e) {
  if (e == cudaSuccess) return IE_OK;
  return e == cudaErrorMemoryAllocation ? IE_ERR_OOM : IE_ERR_CUDA;
}
}  // namespace

#define CK(x)                                       \
  do {                                              \
    cudaError_t e_ = (x);                           \
    if (e_ != cudaSuccess) return map_err(e_);      \
  } while (0)
#define CKS(x)                     \
  do {                             \
    ie_status s_ = (x);            \
    if (s_ != IE_OK) return s_;    \
  } while (0)

// Relative accuracy asked of a mixed-precision G-application outside the relaxed GMRES steps:
// about 9 units of FP64 rounding, so refinement runs until it reaches the FP64 floor.
constexpr double kRefineFull = 1e-15;

struct ie_handle_s {
  int dev = 0;
  int64_t n = 0, n_pad = 0;
  int kl = 0, kv = 0, ldab = 0, ndiag = 0;
  int64_t offsets[IE_MAX_DIAG] = {};
  DiaDev P{};
  cplx* d_A = nullptr;
  cplx* d_B = nullptr;
  zc center;
  double radius = 0;
  int p = 0, q = 0;
  ie_opts opts{};
  zc sigma;
  double normA = 0, normB = 0;
  std::vector<zc> poles, weights;
  cplx* d_poles = nullptr;
  cplx* d_weights = nullptr;
  // factors
  cplx* AB = nullptr;
  int* piv = nullptr;
  cplx* dinv = nullptr;
  cplx* L64 = nullptr;     // q * n_pad * kl: split complex128 L multipliers
  cplx* U64 = nullptr;     // q * n_pad * kv: split complex128 U columns
  cplx* Tb = nullptr;      // q * npanel * 256: forward block transforms
  int* Hb = nullptr;       // q * npanel * 16: their member rows
  cplx* Uinvb = nullptr;   // q * npanel * 64: inverses of U's 8x8 diagonal blocks
  float2* T32 = nullptr;   // complex64 copies (precision = 1)
  float2* Ub32 = nullptr;
  // adjoint pencil (opts.adjoint = 1): (A^H, B^H), conjugated coefficients, U by rows and
  // the per-panel transforms of the conjugate-transpose L sweep
  bool adj = false;
  int side = 0;            // 0: (A, B) on D(c, r); 1: (A^H, B^H) on D(conj c, r)
  DiaDev PH{};
  cplx* d_AH = nullptr;
  cplx* d_BH = nullptr;
  cplx* d_pconj = nullptr;
  cplx* d_wconj = nullptr;
  double normAH = 0, normBH = 0;
  cplx* Ut64 = nullptr;    // q * n_pad * kv
  cplx* Madj64 = nullptr;  // q * npanel * 384
  float2* Ut32 = nullptr;
  float2* Madj32 = nullptr;
  double* d_grad = nullptr;   // n, ie_eig_sensitivity staging (allocated on first use)
  const DiaDev& pen() const { return side ? PH : P; }
  zc ctr() const { return side ? std::conj(center) : center; }
  zc sig() const { return side ? std::conj(sigma) : sigma; }
  double nA() const { return side ? normAH : normA; }
  double nB() const { return side ? normBH : normB; }
  unsigned* bar = nullptr;     // band LU: ring flags (q * ring slots)
  cplx* lu_ring = nullptr;     // band LU: published multipliers (q * slots * (kl + 1))
  int* lu_ring_tp = nullptr;   // band LU: published pivot offsets
  int* status = nullptr;
  int lu_ctas = 0;
  // mixed precision (opts.precision = 1): complex64 factors and FP32-solve scratch
  int precision = 0, refine = 8, klp = 0;
  // Refinement control (see apply_G_mixed): the relative accuracy the next G-application
  // needs (0: as accurate as FP64 refinement gets), the last measured relative error of the
  // plain FP32 solve and the last measured contraction per refinement step (< 0: unknown).
  double refine_target = 1e-15;
  double ref_eps0 = -1.0, ref_c = -1.0;
  unsigned* d_rnrm = nullptr;   // q * kmax * 2: correction / solution maxima (float bits)
  std::vector<unsigned> h_rnrm;
  int64_t refine_solves = 0;
  double refine_last_corr = 0.0;
  float2* AB32 = nullptr;  // complex64 band LU (precision = 1), released after the split copy
  float2* diag32 = nullptr; // q * n_pad: U(j, j) of the complex64 LU (ie_get_factor)
  float2* L32 = nullptr;   // q * n_pad * klp
  float2* U32 = nullptr;   // q * n_pad * kv
  float2* dinv32 = nullptr;
  float2* Y32 = nullptr;   // q * n * kmax
  float2* R32 = nullptr;   // q * n * kmax
  float2* BV32 = nullptr;  // n * kmax
  // workspaces
  int kmax = 0, m_max = 0;
  cplx* Xp = nullptr;     // q * n * kmax
  cplx* BVw = nullptr;    // n * kmax
  cplx* Wb = nullptr;     // n * kmax
  cplx* Yb = nullptr;     // n * kmax  (current block / host staging)
  cplx* Ub = nullptr;     // n * kmax
  cplx* Vh = nullptr;     // HSRR V
  cplx* AVh = nullptr;
  cplx* BVh = nullptr;
  cplx* Wh = nullptr;
  cplx* Xh = nullptr;
  cplx* Ah = nullptr;     // k*k
  cplx* Bh = nullptr;
  cplx* Zq = nullptr;     // 2*k*k
  cplx* Mq = nullptr;     // k*k
  cplx* alpha = nullptr;  // k
  cplx* betaq = nullptr;
  cplx* d_lam = nullptr;
  int* d_perm = nullptr;
  int* d_flags = nullptr;
  double* d_rn = nullptr;  // 3*k
  // Krylov
  KrylovDev K{};
  int* d_act = nullptr;
  int64_t* d_off = nullptr;
  double* d_res = nullptr;
  cplx* hbuf = nullptr;
  double* scratch = nullptr;
  // Givens / combine (sized for nshift_cap shifts)
  int nshift_cap = 0;
  cplx* rot_c = nullptr;
  cplx* rot_s = nullptr;
  cplx* gvec = nullptr;
  cplx* Rscr = nullptr;
  cplx* zbuf = nullptr;
  cplx* d_shifts = nullptr;
  cplx* d_cw = nullptr;
  // host mirrors
  std::vector<int> jc_h;
  std::vector<double> beta_h;
  std::vector<char> conv_h;
  ie_stats stats{};
  int64_t g_columns = 0;
  // band-solve launch timing: event pairs pending until the next stream synchronisation
  struct SolveRec { cudaEvent_t a, b; double flops, bytes; int fp32, adj; };
  std::vector<SolveRec> pending;
  std::vector<cudaEvent_t> event_pool;
  int64_t solve_launches = 0, solve32_launches = 0, adj_launches = 0;
  double t_solve_ms = 0, solve_flops = 0, solve_bytes = 0, t_solve32_ms = 0, solve32_flops = 0;
  double t_adj_ms = 0, adj_flops = 0;
  cudaEvent_t get_event() {
    if (!event_pool.empty()) { cudaEvent_t e = event_pool.back(); event_pool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
  }
  uint32_t salt = 1;
  std::vector<void*> allocs;

  template <typename T>
  cudaError_t alloc(T** p_, size_t count) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    allocs.push_back(v);
    *p_ = (T*)v;
    return cudaSuccess;
  }
  void release(void* p_) {
    if (!p_) return;
    auto it = std::find(allocs.begin(), allocs.end(), p_);
    if (it != allocs.end()) allocs.erase(it);
    cudaFree(p_);
  }
  ~ie_handle_s() {
    for (auto& r : pending) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    for (auto e : event_pool) cudaEventDestroy(e);
    for (void* v : allocs) cudaFree(v);
  }
};

static void fill_solve_stats(ie_handle h, ie_stats* out);

extern "C" void ie_opts_default(ie_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->k = 16;
  o->driver = 1;
  o->m_max = 100;
  o->max_outer = 10;
  o->tau_g = 1e-2;
  o->tau = 1e-10;
  o->gmres_tol = 1e-12;
  o->sigma_is_center = 1;
  o->seed = 0;
  o->precision = 0;
  o->refine_steps = 8;
  o->adjoint = 0;
}

extern "C" const char* ie_status_str(ie_status s) {
  switch (s) {
    case IE_OK: return "IE_OK";
    case IE_ERR_ARG: return "IE_ERR_ARG: invalid argument";
    case IE_ERR_CUDA: return "IE_ERR_CUDA: CUDA error";
    case IE_ERR_OOM: return "IE_ERR_OOM: device allocation failed";
    case IE_ERR_SINGULAR: return "IE_ERR_SINGULAR: zero pivot in the band LU";
    case IE_ERR_NOCONV: return "IE_ERR_NOCONV: iteration limit reached";
    case IE_ERR_BREAKDOWN: return "IE_ERR_BREAKDOWN: orthogonalisation breakdown";
    case IE_ERR_TIMEOUT: return "IE_ERR_TIMEOUT: a device-side bounded wait gave up";
    case IE_ERR_SCRATCH_LIMIT:
      return "IE_ERR_SCRATCH_LIMIT: (q+1)*n*k complex128 values exceed IE_STATIC_SCRATCH_BYTES";
  }
  return "unknown ie_status";
}

// ------------------------------ coefficients --------------------------------------------------
// Eq. (pwtp): p_i = c + r e^{i theta_i}, w_i = r e^{i theta_i} / q, theta_i = (2i-1) pi / q.
static void inner_coeffs(zc c, double r, int q, std::vector<zc>& poles, std::vector<zc>& w) {
  poles.resize(q);
  w.resize(q);
  for (int i = 1; i <= q; ++i) {
    const double th = (2.0 * i - 1.0) * M_PI / q;
    const zc e(std::cos(th), std::sin(th));
    poles[i - 1] = c + r * e;
    w[i - 1] = r * e / (double)q;
  }
}
// Thm 2: sigma_j = e^{i (2j-1) pi / p}; s_j = 1/(1+sigma_j); c_j = -(1/p) sigma_j/(1+sigma_j);
// for odd p the root sigma = -1 (j = (p+1)/2) is left out and contributes (1/p) R_q.
static void outer_coeffs(int p, std::vector<zc>& s, std::vector<zc>& cw, double& odd) {
  s.clear();
  cw.clear();
  odd = (p % 2) ? 1.0 / p : 0.0;
  for (int j = 1; j <= p; ++j) {
    if ((p % 2) && j == (p + 1) / 2) continue;
    const double th = (2.0 * j - 1.0) * M_PI / p;
    const zc sg(std::cos(th), std::sin(th));
    s.push_back(1.0 / (1.0 + sg));
    cw.push_back(-(1.0 / p) * sg / (1.0 + sg));
  }
}

// ------------------------------ workspace -------------------------------------------------------
static ie_status ensure_shift_capacity(ie_handle h, int nshift) {
  if (nshift <= h->nshift_cap) return IE_OK;
  int cap = std::max(nshift, 2 * h->nshift_cap);
  const int64_t k = h->kmax, M = h->m_max;
  for (void* p_ : {(void*)h->rot_c, (void*)h->rot_s, (void*)h->gvec, (void*)h->Rscr,
                   (void*)h->zbuf, (void*)h->d_shifts, (void*)h->d_cw})
    h->release(p_);
  CK(h->alloc(&h->rot_c, (size_t)(k * cap * M)));
  CK(h->alloc(&h->rot_s, (size_t)(k * cap * M)));
  CK(h->alloc(&h->gvec, (size_t)(k * cap * (M + 1))));
  CK(h->alloc(&h->Rscr, (size_t)(k * cap * M * M)));
  CK(h->alloc(&h->zbuf, (size_t)(2 * k * cap * M + k * cap * (M + 1) + k * (M + 1))));
  CK(h->alloc(&h->d_shifts, (size_t)cap));
  CK(h->alloc(&h->d_cw, (size_t)cap));
  h->nshift_cap = cap;
  return IE_OK;
}

static ie_status alloc_workspace(ie_handle h) {
  const int64_t n = h->n, k = h->kmax, M = h->m_max, q = h->q;
  CK(h->alloc(&h->Xp, (size_t)(q * n * k)));
  CK(h->alloc(&h->BVw, (size_t)(n * k)));
  CK(h->alloc(&h->Wb, (size_t)(n * k)));
  CK(h->alloc(&h->Yb, (size_t)(n * k)));
  CK(h->alloc(&h->Ub, (size_t)(n * k)));
  CK(h->alloc(&h->Vh, (size_t)(n * k)));
  CK(h->alloc(&h->AVh, (size_t)(n * k)));
  CK(h->alloc(&h->BVh, (size_t)(n * k)));
  CK(h->alloc(&h->Wh, (size_t)(n * k)));
  CK(h->alloc(&h->Xh, (size_t)(n * k)));
  CK(h->alloc(&h->Ah, (size_t)(k * k)));
  CK(h->alloc(&h->Bh, (size_t)(k * k)));
  CK(h->alloc(&h->Zq, (size_t)(2 * k * k)));
  CK(h->alloc(&h->Mq, (size_t)(k * k)));
  CK(h->alloc(&h->alpha, (size_t)k));
  CK(h->alloc(&h->betaq, (size_t)k));
  CK(h->alloc(&h->d_lam, (size_t)k));
  CK(h->alloc(&h->d_perm, (size_t)k));
  CK(h->alloc(&h->d_flags, (size_t)k));
  CK(h->alloc(&h->d_rn, (size_t)(3 * k)));
  // Krylov bases
  CK(h->alloc(&h->K.V, (size_t)(k * (M + 1) * n)));
  CK(h->alloc(&h->K.H, (size_t)(k * (M + 1) * M)));
  CK(h->alloc(&h->K.beta, (size_t)k));
  CK(h->alloc(&h->K.jc, (size_t)k));
  CK(h->alloc(&h->K.brk, (size_t)k));
  h->K.n = n;
  h->K.m_max = (int)M;
  CK(cudaMemset(h->K.H, 0, sizeof(cplx) * (size_t)(k * (M + 1) * M)));
  CK(h->alloc(&h->d_act, (size_t)k));
  CK(h->alloc(&h->d_off, (size_t)k));
  CK(h->alloc(&h->d_res, (size_t)k));
  const int64_t LD = M + 2;
  CK(h->alloc(&h->hbuf, (size_t)(2 * k * LD + k + 3 * (k + 1) + 16)));
  const int64_t nch512 = (n + 511) / 512, nblk = (n + 255) / 256;
  int64_t need = 2 * k * nch512 * LD + k * nblk;                 // Arnoldi partials
  need = std::max<int64_t>(need, 2 * nch512 * k * k);            // Gram partials
  need = std::max<int64_t>(need, 3 * k * nblk);                  // residual partials
  need = std::max<int64_t>(need, 2 * nch512 * (k + 1));          // orth partials
  need = std::max<int64_t>(need, 2 * (k * 64 + k));              // column norms
  CK(h->alloc(&h->scratch, (size_t)(need + 1024)));
  CKS(ensure_shift_capacity(h, std::max(1, h->p)));
  h->jc_h.assign(k, 0);
  h->beta_h.assign(k, 0.0);
  h->conv_h.assign(k, 0);
  return IE_OK;
}

// Adjoint pencil for ie_apply_GH / ie_solve_left, from the band factors (AB or AB32 must still
// be present): (A^H, B^H) and their norms, conj(p_i), conj(w_i), U by rows and the phase-2
// transforms, in the handle's factor precision.
static ie_status setup_adjoint(ie_handle h, cudaStream_t s) {
  const int q = h->q;
  const size_t nd = (size_t)h->ndiag * h->n, np = (size_t)(h->n_pad / 8);
  CK(h->alloc(&h->d_AH, nd));
  CK(h->alloc(&h->d_BH, nd));
  launch_dia_adjoint(h->P, h->d_AH, h->d_BH, &h->PH, s);
  double* dn = nullptr;
  CK(h->alloc(&dn, 2));
  launch_norm1_cols(h->PH, 0, dn, nullptr, s);
  launch_norm1_cols(h->PH, 1, dn + 1, nullptr, s);
  double hn[2];
  CK(cudaMemcpyAsync(hn, dn, sizeof(hn), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  h->normAH = hn[0];
  h->normBH = hn[1];
  std::vector<cplx> pc(q), wc(q);
  for (int i = 0; i < q; ++i) {
    pc[i] = to_c(std::conj(h->poles[i]));
    wc[i] = to_c(std::conj(h->weights[i]));
  }
  CK(h->alloc(&h->d_pconj, q));
  CK(h->alloc(&h->d_wconj, q));
  CK(cudaMemcpyAsync(h->d_pconj, pc.data(), sizeof(cplx) * q, cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(h->d_wconj, wc.data(), sizeof(cplx) * q, cudaMemcpyHostToDevice, s));
  const size_t nu = (size_t)q * h->n_pad * h->kv, nm = (size_t)q * np * 384;
  if (h->precision == 0) {
    CK(h->alloc(&h->Ut64, nu));
    CK(h->alloc(&h->Madj64, nm));
  } else {
    CK(h->alloc(&h->Ut32, nu));
    CK(h->alloc(&h->Madj32, nm));
  }
  if (h->precision == 0) {
    launch_u_rows(q, h->n, h->n_pad, h->kl, h->ldab, h->AB, h->Ut64, nullptr, s);
    launch_adj_transforms(q, h->n, h->n_pad, h->kl, h->ldab, h->AB, h->piv, h->Hb, h->Madj64,
                          nullptr, s);
  } else {
    launch_u_rows(q, h->n, h->n_pad, h->kl, h->ldab, h->AB32, h->Ut32, s);
    launch_adj_transforms(q, h->n, h->n_pad, h->kl, h->ldab, h->AB32, h->piv, h->Hb, h->Madj32, s);
  }
  CK(cudaStreamSynchronize(s));
  h->adj = true;
  return IE_OK;
}

// ------------------------------ create / destroy -------------------------------------------------
extern "C" ie_status ie_create(const ie_pencil* pen, ie_complex center, double radius, int32_t p,
                               int32_t q, const ie_opts* opts_in, void* stream, ie_handle* out) {
  if (!pen || !out || !pen->h_offsets || !pen->d_A_dia || !pen->d_B_dia) return IE_ERR_ARG;
  *out = nullptr;
  ie_opts opts;
  if (opts_in) opts = *opts_in; else ie_opts_default(&opts);
  if (pen->n < 2 || pen->ndiag < 1 || pen->ndiag > IE_MAX_DIAG) return IE_ERR_ARG;
  if (p < 1 || q < 1 || !(radius > 0.0) || !std::isfinite(radius)) return IE_ERR_ARG;
  if (opts.k < 1 || opts.k > pen->n || opts.m_max < 1 || opts.m_max > 1000 ||
      opts.max_outer < 1 || (opts.driver != 1 && opts.driver != 2))
    return IE_ERR_ARG;
  if (!(opts.gmres_tol > 0) || !(opts.tau > 0) || !(opts.tau_g > 0)) return IE_ERR_ARG;
  if ((opts.precision != 0 && opts.precision != 1) || opts.refine_steps < 0 ||
      opts.refine_steps > 20 || (opts.adjoint != 0 && opts.adjoint != 1))
    return IE_ERR_ARG;
  int kl = 0;
  for (int d = 0; d < pen->ndiag; ++d) {
    const int64_t o = pen->h_offsets[d];
    if (o <= -pen->n || o >= pen->n) return IE_ERR_ARG;
    kl = (int)std::max<int64_t>(kl, o < 0 ? -o : o);
  }
  if (kl < 1 || 2 * kl + 8 > 1152) return IE_ERR_ARG;   // band solve supports half bandwidth <= 572
  cudaStream_t s = (cudaStream_t)stream;
  ie_handle h = new ie_handle_s();
  cudaGetDevice(&h->dev);
  h->n = pen->n;
  h->n_pad = (pen->n + 7) / 8 * 8;   // whole 8-column factor panels
  h->kl = kl;
  h->kv = 2 * kl;
  h->ldab = 3 * kl + 1;
  h->ndiag = pen->ndiag;
  h->center = to_z(center);
  h->radius = radius;
  h->p = p;
  h->q = q;
  h->opts = opts;
  h->kmax = opts.k;
  h->m_max = opts.m_max;
  h->sigma = opts.sigma_is_center ? h->center : zc(opts.sigma_re, opts.sigma_im);
  h->precision = opts.precision;
  h->refine = opts.refine_steps;
  h->klp = kl + (kl & 1);
  auto fail = [&](ie_status st) { delete h; return st; };
  const size_t dia_bytes = sizeof(cplx) * (size_t)pen->ndiag * (size_t)pen->n;
  if (h->alloc(&h->d_A, (size_t)pen->ndiag * pen->n) != cudaSuccess) return fail(IE_ERR_OOM);
  if (h->alloc(&h->d_B, (size_t)pen->ndiag * pen->n) != cudaSuccess) return fail(IE_ERR_OOM);
  if (cudaMemcpyAsync(h->d_A, pen->d_A_dia, dia_bytes, cudaMemcpyDefault, s) != cudaSuccess ||
      cudaMemcpyAsync(h->d_B, pen->d_B_dia, dia_bytes, cudaMemcpyDefault, s) != cudaSuccess)
    return fail(IE_ERR_CUDA);
  h->P.n = h->n;
  h->P.ndiag = h->ndiag;
  for (int d = 0; d < h->ndiag; ++d) h->P.off[d] = h->offsets[d] = pen->h_offsets[d];
  h->P.A = h->d_A;
  h->P.B = h->d_B;
  // coefficients
  inner_coeffs(h->center, radius, q, h->poles, h->weights);
  std::vector<cplx> tmp(q);
  if (h->alloc(&h->d_poles, q) != cudaSuccess || h->alloc(&h->d_weights, q) != cudaSuccess)
    return fail(IE_ERR_OOM);
  for (int i = 0; i < q; ++i) tmp[i] = to_c(h->poles[i]);
  cudaMemcpyAsync(h->d_poles, tmp.data(), sizeof(cplx) * q, cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);
  for (int i = 0; i < q; ++i) tmp[i] = to_c(h->weights[i]);
  cudaMemcpyAsync(h->d_weights, tmp.data(), sizeof(cplx) * q, cudaMemcpyHostToDevice, s);
  cudaStreamSynchronize(s);
  // norms ||A||_1, ||B||_1
  double* dn = nullptr;
  if (h->alloc(&dn, 2) != cudaSuccess) return fail(IE_ERR_OOM);
  launch_norm1_cols(h->P, 0, dn, nullptr, s);
  launch_norm1_cols(h->P, 1, dn + 1, nullptr, s);
  double hn[2];
  if (cudaMemcpyAsync(hn, dn, sizeof(hn), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail(IE_ERR_CUDA);
  h->normA = hn[0];
  h->normB = hn[1];
  // factors: complex128 band LU (precision 0), or the same LU in complex64 with FP32
  // arithmetic (precision 1), from K_i assembled in the factor precision
  const bool mixed = opts.precision == 1;
  const size_t nab = (size_t)q * h->n_pad * h->ldab;
  if ((mixed ? h->alloc(&h->AB32, nab) : h->alloc(&h->AB, nab)) != cudaSuccess ||
      h->alloc(&h->piv, (size_t)q * h->n_pad) != cudaSuccess ||
      (mixed ? h->alloc(&h->dinv32, (size_t)q * h->n_pad)
             : h->alloc(&h->dinv, (size_t)q * h->n_pad)) != cudaSuccess ||
      h->alloc(&h->lu_ring, band_lu_ring_elems(q, kl)) != cudaSuccess ||
      h->alloc(&h->lu_ring_tp, band_lu_ring_ints(q)) != cudaSuccess ||
      h->alloc(&h->bar, (size_t)q * band_lu_ring_slots(q)) != cudaSuccess ||
      h->alloc(&h->status, ST_COUNT) != cudaSuccess)
    return fail(IE_ERR_OOM);
  cudaMemsetAsync(h->status, 0, sizeof(int) * ST_COUNT, s);
  cudaMemsetAsync(h->piv, 0, sizeof(int) * (size_t)q * h->n_pad, s);
  if (mixed) cudaMemsetAsync(h->dinv32, 0, sizeof(float2) * (size_t)q * h->n_pad, s);
  else cudaMemsetAsync(h->dinv, 0, sizeof(cplx) * (size_t)q * h->n_pad, s);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  cudaError_t le;
  if (mixed) {
    launch_assemble(h->P, h->d_poles, q, kl, h->ldab, h->n_pad, h->AB32, s);
    le = launch_band_lu(q, h->n, kl, h->ldab, h->n_pad, h->AB32, h->piv, h->dinv32,
                        (float2*)h->lu_ring, h->lu_ring_tp, h->bar, band_lu_ring_slots(q),
                        h->status, s, &h->lu_ctas);
  } else {
    launch_assemble(h->P, h->d_poles, q, kl, h->ldab, h->n_pad, h->AB, s);
    le = launch_band_lu(q, h->n, kl, h->ldab, h->n_pad, h->AB, h->piv, h->dinv, h->lu_ring,
                        h->lu_ring_tp, h->bar, band_lu_ring_slots(q), h->status, s, &h->lu_ctas);
  }
  cudaEventRecord(e1, s);
  if (le != cudaSuccess) { cudaEventDestroy(e0); cudaEventDestroy(e1); return fail(map_err(le)); }
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaEventDestroy(e0); cudaEventDestroy(e1);
    return fail(IE_ERR_CUDA);
  }
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->stats.t_factor_ms = ms;
  int st[ST_COUNT];
  cudaMemcpy(st, h->status, sizeof(st), cudaMemcpyDeviceToHost);
  if (st[ST_TIMEOUT]) return fail(IE_ERR_TIMEOUT);
  {
    const size_t np = (size_t)(h->n_pad / 8);
    if (!mixed) {
      if (h->alloc(&h->L64, (size_t)q * h->n_pad * kl) != cudaSuccess ||
          h->alloc(&h->U64, (size_t)q * h->n_pad * h->kv) != cudaSuccess ||
          h->alloc(&h->Tb, (size_t)q * np * 256) != cudaSuccess ||
          h->alloc(&h->Hb, (size_t)q * np * 16) != cudaSuccess ||
          h->alloc(&h->Uinvb, (size_t)q * np * 64) != cudaSuccess)
        return fail(IE_ERR_OOM);
      launch_factors_split64(q, h->n_pad, kl, h->ldab, h->AB, h->L64, h->U64, s);
      launch_block_transforms(q, h->n, h->n_pad, kl, h->ldab, h->AB, h->piv, h->dinv, h->Tb,
                              h->Hb, h->Uinvb, nullptr, nullptr, s);
    } else {
      if (h->alloc(&h->L32, (size_t)q * h->n_pad * h->klp) != cudaSuccess ||
          h->alloc(&h->U32, (size_t)q * h->n_pad * h->kv) != cudaSuccess ||
          h->alloc(&h->diag32, (size_t)q * h->n_pad) != cudaSuccess ||
          h->alloc(&h->Hb, (size_t)q * np * 16) != cudaSuccess ||
          h->alloc(&h->T32, (size_t)q * np * 256) != cudaSuccess ||
          h->alloc(&h->Ub32, (size_t)q * np * 64) != cudaSuccess)
        return fail(IE_ERR_OOM);
      launch_factors_split32(q, h->n_pad, kl, h->ldab, h->klp, h->AB32, h->L32, h->U32,
                             h->diag32, s);
      launch_block_transforms(q, h->n, h->n_pad, kl, h->ldab, h->AB32, h->piv, h->dinv32, h->Hb,
                              h->T32, h->Ub32, s);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return fail(IE_ERR_CUDA);
    if (opts.adjoint) {
      ie_status as = setup_adjoint(h, s);
      if (as != IE_OK) return fail(as);
    }
  }
  ie_status ws = alloc_workspace(h);
  if (ws != IE_OK) return fail(ws);
  if (mixed) {
    const size_t nk = (size_t)h->n * h->kmax;
    if (h->alloc(&h->Y32, (size_t)q * nk) != cudaSuccess ||
        h->alloc(&h->R32, (size_t)q * nk) != cudaSuccess ||
        h->alloc(&h->BV32, nk) != cudaSuccess ||
        h->alloc(&h->d_rnrm, (size_t)q * h->kmax * 2) != cudaSuccess)
      return fail(IE_ERR_OOM);
    h->h_rnrm.assign((size_t)q * h->kmax * 2, 0u);
    // the band storage of the complex64 LU is no longer used: the split copy serves the solves
    h->release(h->AB32);
    h->AB32 = nullptr;
  }
  if (cudaGetLastError() != cudaSuccess) return fail(IE_ERR_CUDA);
  *out = h;
  return st[ST_SINGULAR] ? IE_ERR_SINGULAR : IE_OK;
}

extern "C" ie_status ie_destroy(ie_handle h) {
  if (!h) return IE_ERR_ARG;
  delete h;
  return IE_OK;
}

// ------------------------------ host/device staging ----------------------------------------------
static ie_status stage_in(ie_handle h, const ie_complex* src, int64_t ld, int k, cplx* dst,
                          cudaStream_t s, const cplx** out) {
  if (is_device_ptr(src)) {
    *out = (const cplx*)src;
    return IE_OK;
  }
  CK(cudaMemcpy2DAsync(dst, sizeof(cplx) * h->n, src, sizeof(cplx) * ld, sizeof(cplx) * h->n, k,
                       cudaMemcpyHostToDevice, s));
  *out = dst;
  return IE_OK;
}
static ie_status stage_out(ie_handle h, const cplx* src, int64_t lds, int k, ie_complex* dst,
                           int64_t ldd, cudaStream_t s) {
  if ((const void*)src == (const void*)dst) return IE_OK;
  CK(cudaMemcpy2DAsync(dst, sizeof(cplx) * ldd, src, sizeof(cplx) * lds, sizeof(cplx) * h->n, k,
                       cudaMemcpyDefault, s));
  return IE_OK;
}
// Accumulates the device time of band-solve launches whose events have completed
// (called after a stream synchronisation).
static void flush_solve_timing(ie_handle h) {
  std::vector<ie_handle_s::SolveRec> keep;
  for (auto& r : h->pending) {
    if (cudaEventQuery(r.b) != cudaSuccess) { cudaGetLastError(); keep.push_back(r); continue; }
    float ms = 0;
    cudaEventElapsedTime(&ms, r.a, r.b);
    if (r.adj) {
      h->t_adj_ms += ms;
      h->adj_flops += r.flops;
      h->adj_launches += 1;
    } else if (r.fp32) {
      h->t_solve32_ms += ms;
      h->solve32_flops += r.flops;
      h->solve32_launches += 1;
    } else {
      h->t_solve_ms += ms;
      h->solve_flops += r.flops;
      h->solve_bytes += r.bytes;
      h->solve_launches += 1;
    }
    h->event_pool.push_back(r.a);
    h->event_pool.push_back(r.b);
  }
  h->pending.swap(keep);
}

static ie_status check_status(ie_handle h, cudaStream_t s) {
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  flush_solve_timing(h);
  int st[ST_COUNT];
  CK(cudaMemcpy(st, h->status, sizeof(st), cudaMemcpyDeviceToHost));
  if (st[ST_TIMEOUT]) return IE_ERR_TIMEOUT;
  return IE_OK;
}

// ------------------------------ inner operator G ----------------------------------------------
// GV = sum_i w_i K_i^{-1} B V (Eq. linearsolve2). V columns at V + off[c] when d_off != null.
// On the adjoint side (h->side = 1): GV = sum_i conj(w_i) K_i^{-H} B^H V.
static ie_status apply_G_mixed(ie_handle h, int k, cplx* GV, int64_t ldg, cudaStream_t s);

static ie_status apply_G_dev(ie_handle h, const cplx* V, int64_t ldv, const int64_t* d_off, int k,
                             cplx* GV, int64_t ldg, cudaStream_t s) {
  if (k <= 0) return IE_OK;
  launch_spmv(h->pen(), make_double2(0, 0), make_double2(1, 0), V, ldv, d_off, k, h->BVw, h->n, s);
  if (h->precision == 1) return apply_G_mixed(h, k, GV, ldg, s);
  ie_handle_s::SolveRec rec;
  rec.a = h->get_event();
  rec.b = h->get_event();
  {
    // algorithmic work of one launch: forward n*kl and backward n*kv complex FMAs per (pole,
    // column) less the band corners, plus two complex products per row (1/u_jj and w_i)
    const double n = (double)h->n, kl = h->kl, kv = h->kv, q = h->q;
    const double fwd = n * kl - 0.5 * kl * (kl + 1), bwd = n * kv - 0.5 * kv * (kv + 1);
    rec.flops = q * k * (8.0 * (fwd + bwd) + 12.0 * n);
    rec.bytes = q * n * (16.0 * (kl + kv + 1) + 4.0) + 16.0 * n * k * (1.0 + 3.0 * q);
    rec.fp32 = 0;
    rec.adj = h->side;
  }
  cudaEventRecord(rec.a, s);
  if (h->side) {
    CK(launch_band_solve_adj(h->q, h->n, h->kl, h->n_pad, h->L64, h->Ut64, h->Uinvb, h->Madj64,
                             h->Hb, h->d_wconj, h->BVw, h->n, k, h->Xp, h->n,
                             h->n * (int64_t)h->kmax, h->status, s));
  } else {
    CK(launch_band_solve(h->q, h->n, h->kl, h->n_pad, h->L64, h->U64, h->piv, h->dinv, h->Tb,
                         h->Hb, h->Uinvb, h->d_weights, h->BVw, h->n, k, h->Xp, h->n,
                         h->n * (int64_t)h->kmax, h->status, s));
  }
  cudaEventRecord(rec.b, s);
  h->pending.push_back(rec);
  launch_pole_sum(h->q, h->n, k, h->Xp, h->n, h->n * (int64_t)h->kmax, GV, ldg, s);
  h->g_columns += k;
  return IE_OK;
}

// Mixed precision (opts.precision = 1), B V already in h->BVw: per pole i,
//   x_i = K~_i^{-1} BV (complex64 factors, FP32 solve), then FP64 iterative refinement
//   x_i += K~_i^{-1} (BV - K_i x_i), with the residual formed in FP64 from the DIA pencil;
//   GV = sum_i w_i x_i in FP64.
// The adjoint side uses K_i^H = conj(p_i) B^H - A^H and conj(w_i) throughout.
//
// The number of refinement steps is measured, not fixed. After step t the largest relative
// correction d_t = max_{i,c} |dx_{i,c}|_inf / |x_{i,c}|_inf estimates the error that step
// removed; refinement contracts the error by about c = d_t / d_{t-1} per step, so the error
// left is about c d_t. The steps stop when that estimate is at most h->refine_target, when
// the corrections stop shrinking (d_t > d_{t-1} / 2: the FP64 residual's own rounding floor),
// or after opts.refine_steps steps. The GMRES loop passes larger targets as its residual falls
// (relaxation, see filter_dev). When
// the last application measured a plain-solve error eps0 with 10 eps0 <= target, no step is
// taken. Outside the relaxed GMRES steps the target is kRefineFull.
static ie_status apply_G_mixed(ie_handle h, int k, cplx* GV, int64_t ldg, cudaStream_t s) {
  const int64_t n = h->n, ps = n * (int64_t)h->kmax;
  const double nn = (double)n, kl = h->kl, kv = h->kv, q = h->q;
  const double fwd = nn * kl - 0.5 * kl * (kl + 1), bwd = nn * kv - 0.5 * kv * (kv + 1);
  const double flops = q * k * (8.0 * (fwd + bwd) + 12.0 * nn);
  const bool adj = h->side != 0;
  const double target = h->refine_target;
  auto solve = [&](int it) -> ie_status {
    ie_handle_s::SolveRec rec;
    rec.a = h->get_event();
    rec.b = h->get_event();
    rec.flops = flops;
    rec.bytes = 0;
    rec.fp32 = 1;
    rec.adj = adj;
    cudaEventRecord(rec.a, s);
    const float2* rhs = it == 0 ? h->BV32 : h->R32;
    const int64_t rstride = it == 0 ? 0 : ps;
    // it = 0: X = K~^{-1} BV; it > 0: the correction K~^{-1} r in place into Y32
    if (adj) {
      CK(launch_band_solve_adj32(h->q, n, h->kl, h->n_pad, h->L32, h->klp, h->Ut32, h->Ub32,
                                 h->Madj32, h->Hb, h->d_wconj, rhs, n, rstride, k, h->Y32, n, ps,
                                 h->Xp, n, ps, it > 0 ? 1 : 0, h->status, s));
    } else {
      CK(launch_band_solve32(h->q, n, h->kl, h->n_pad, h->L32, h->klp, h->U32, h->kv, h->piv,
                             h->dinv32, h->T32, h->Hb, h->Ub32, h->d_weights, rhs, n, rstride, k,
                             h->Y32, n, ps, h->Xp, n, ps, it > 0 ? 1 : 0, h->status, s));
    }
    cudaEventRecord(rec.b, s);
    h->pending.push_back(rec);
    return IE_OK;
  };
  launch_to_c64(n, k, h->BVw, n, h->BV32, n, s);
  CKS(solve(0));
  const bool skip = h->ref_eps0 > 0.0 && 10.0 * h->ref_eps0 <= target;
  double prev = -1.0, last = 0.0;
  const size_t nn2 = (size_t)h->q * k * 2;
  for (int it = 1; it <= h->refine && !skip; ++it) {
    launch_pole_residual(h->pen(), adj ? h->d_pconj : h->d_poles, h->q, k, h->BVw, n, h->Xp, n,
                         ps, h->R32, n, ps, s);
    CKS(solve(it));
    CK(cudaMemsetAsync(h->d_rnrm, 0, sizeof(unsigned) * nn2, s));
    launch_refine_add(h->q, n, k, h->Y32, n, ps, h->Xp, n, ps, h->d_rnrm, s);
    CK(cudaMemcpyAsync(h->h_rnrm.data(), h->d_rnrm, sizeof(unsigned) * nn2, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    h->refine_solves += 1;
    double d = 0.0;
    for (size_t e = 0; e < nn2; e += 2) {
      float dm, xm;
      std::memcpy(&dm, &h->h_rnrm[e], sizeof(float));
      std::memcpy(&xm, &h->h_rnrm[e + 1], sizeof(float));
      if (xm > 0.0f) d = std::max(d, (double)dm / (double)xm);
    }
    last = d;
    if (it == 1) h->ref_eps0 = d;
    if (prev > 0.0) {
      if (d > 0.5 * prev) break;                 // no longer shrinking: the FP64 floor
      h->ref_c = std::min(1.0, d / prev);
    }
    const double c = prev > 0.0 ? d / prev : (h->ref_c > 0.0 ? 10.0 * h->ref_c : 1.0);
    if (d * std::min(1.0, c) <= target) break;
    prev = d;
  }
  h->refine_last_corr = last;
  launch_pole_wsum(h->q, n, k, h->Xp, n, ps, adj ? h->d_wconj : h->d_weights, GV, ldg, s);
  h->g_columns += k;
  return IE_OK;
}

// ------------------------------ filter (multi-shift GMRES) -----------------------------------
// U = sum_j c_j (s_j I - G)^{-1} Ytilde (+ odd Ytilde). With reuse, the Krylov spaces of the
// previous call are kept and only extended (Alg. 2).
static ie_status filter_dev(ie_handle h, const cplx* Y, int64_t ldy, int k, cplx* U, int64_t ldu,
                            int p_use, bool reuse, cudaStream_t s, bool* noconv) {
  const int64_t n = h->n;
  *noconv = false;
  if (!reuse) {
    CKS(apply_G_dev(h, Y, ldy, nullptr, k, h->Wb, n, s));      // Ytilde = G(Y)
    launch_krylov_start(h->K, k, h->Wb, n, h->scratch, s);
    CK(cudaMemcpyAsync(h->beta_h.data(), h->K.beta, sizeof(double) * k, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int c = 0; c < k; ++c) h->jc_h[c] = 0;
  }
  std::vector<zc> sh, cw;
  double odd = 0;
  outer_coeffs(p_use, sh, cw, odd);
  const int nshift = (int)sh.size();
  CKS(ensure_shift_capacity(h, std::max(nshift, 1)));
  {
    std::vector<cplx> a(nshift), b(nshift);
    for (int i = 0; i < nshift; ++i) { a[i] = to_c(sh[i]); b[i] = to_c(cw[i]); }
    if (nshift) {
      CK(cudaMemcpyAsync(h->d_shifts, a.data(), sizeof(cplx) * nshift, cudaMemcpyHostToDevice, s));
      CK(cudaMemcpyAsync(h->d_cw, b.data(), sizeof(cplx) * nshift, cudaMemcpyHostToDevice, s));
      CK(cudaStreamSynchronize(s));
    }
  }
  const double tol = h->opts.gmres_tol;
  std::vector<int> act;
  std::vector<double> res(k);
  double rmax = 1.0;   // largest relative GMRES residual among the active columns so far
  // convergence state of every column for the current shift set
  for (int c = 0; c < k; ++c) h->conv_h[c] = (h->beta_h[c] > 0.0) ? 0 : 1;
  if (nshift == 0) {
    for (int c = 0; c < k; ++c) h->conv_h[c] = 1;
  } else if (reuse) {
    act.clear();
    for (int c = 0; c < k; ++c)
      if (!h->conv_h[c] && h->jc_h[c] > 0) act.push_back(c);
    if (!act.empty()) {
      CK(cudaMemcpyAsync(h->d_act, act.data(), sizeof(int) * act.size(), cudaMemcpyHostToDevice, s));
      launch_givens(h->K, h->d_act, (int)act.size(), h->d_shifts, nshift, h->rot_c, h->rot_s,
                    h->gvec, 1, h->d_res, s);
      CK(cudaMemcpyAsync(res.data(), h->d_res, sizeof(double) * act.size(), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      rmax = 0.0;
      for (size_t i = 0; i < act.size(); ++i) {
        if (res[i] <= tol) h->conv_h[act[i]] = 1;
        else rmax = std::max(rmax, res[i]);
      }
      if (rmax == 0.0) rmax = 1.0;
    }
  }
  while (true) {
    act.clear();
    for (int c = 0; c < k; ++c)
      if (!h->conv_h[c]) {
        if (h->jc_h[c] >= h->m_max) { *noconv = true; continue; }
        act.push_back(c);
      }
    if (act.empty()) break;
    const int kact = (int)act.size();
    CK(cudaMemcpyAsync(h->d_act, act.data(), sizeof(int) * kact, cudaMemcpyHostToDevice, s));
    launch_active_offsets(h->K, h->d_act, kact, h->d_off, s);
    // Inexact Krylov relaxation (Bouras & Fraysse, SIAM J. Matrix Anal. Appl. 26, 2005;
    // Simoncini & Szyld, SIAM J. Sci. Comput. 25, 2003): an operator error eps at a step whose
    // residual is r changes the final residual by about eps * r, so the mixed-precision path
    // may refine G v_j only to tol / (50 r) (50: a bound on the steps that add such errors).
    if (h->precision == 1) h->refine_target = std::min(1e-2, tol / (50.0 * rmax));
    const ie_status ga = apply_G_dev(h, h->K.V, n, h->d_off, kact, h->Wb, n, s);   // w = G v_j
    h->refine_target = kRefineFull;
    CKS(ga);
    launch_arnoldi_cgs2(h->K, h->d_act, kact, h->Wb, n, h->hbuf, h->scratch, s);
    launch_givens(h->K, h->d_act, kact, h->d_shifts, nshift, h->rot_c, h->rot_s, h->gvec, 0,
                  h->d_res, s);
    CK(cudaMemcpyAsync(res.data(), h->d_res, sizeof(double) * kact, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    flush_solve_timing(h);
    rmax = 0.0;
    for (int i = 0; i < kact; ++i) {
      const int c = act[i];
      h->jc_h[c] += 1;
      if (res[i] <= tol) h->conv_h[c] = 1;
      else rmax = std::max(rmax, res[i]);
    }
  }
  launch_krylov_combine(h->K, k, h->d_shifts, h->d_cw, nshift, odd, h->Rscr, h->zbuf, U, ldu, s);
  int mx = 0, mn = 1 << 30;
  for (int c = 0; c < k; ++c) { mx = std::max(mx, h->jc_h[c]); mn = std::min(mn, h->jc_h[c]); }
  h->stats.gmres_iters_max = mx;
  h->stats.gmres_iters_min = (k > 0) ? mn : 0;
  h->stats.p_final = p_use;
  return check_status(h, s);
}

extern "C" ie_status ie_filter_apply(ie_handle h, const ie_complex* Y_any, int64_t ldy, int32_t k,
                                     ie_complex* U_any, int64_t ldu, void* stream) {
  if (!h || !Y_any || !U_any || k < 1 || k > h->kmax || ldy < h->n || ldu < h->n) return IE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  const cplx* Y;
  CKS(stage_in(h, Y_any, ldy, k, h->Yb, s, &Y));
  const bool udev = is_device_ptr(U_any);
  cplx* U = udev ? (cplx*)U_any : h->Ub;
  const int64_t ldU = udev ? ldu : h->n;
  bool nc = false;
  ie_status st = filter_dev(h, Y, Y == h->Yb ? h->n : ldy, k, U, ldU, h->p, false, s, &nc);
  if (st == IE_OK && !udev) st = stage_out(h, U, ldU, k, U_any, ldu, s);
  cudaEventRecord(e1, s);
  cudaStreamSynchronize(s);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->stats.t_filter_ms = ms;
  h->stats.g_columns = h->g_columns;
  if (st != IE_OK) return st;
  return nc ? IE_ERR_NOCONV : IE_OK;
}

extern "C" ie_status ie_apply_G(ie_handle h, const ie_complex* V_any, int64_t ldv, int32_t k,
                                ie_complex* GV_any, int64_t ldgv, void* stream) {
  if (!h || !V_any || !GV_any || k < 1 || k > h->kmax || ldv < h->n || ldgv < h->n) return IE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const cplx* V;
  CKS(stage_in(h, V_any, ldv, k, h->Yb, s, &V));
  const bool gdev = is_device_ptr(GV_any);
  cplx* G = gdev ? (cplx*)GV_any : h->Ub;
  const int64_t ldG = gdev ? ldgv : h->n;
  CKS(apply_G_dev(h, V, V == h->Yb ? h->n : ldv, nullptr, k, G, ldG, s));
  if (!gdev) CKS(stage_out(h, G, ldG, k, GV_any, ldgv, s));
  h->stats.g_columns = h->g_columns;
  return check_status(h, s);
}

extern "C" ie_status ie_spmv(ie_handle h, int32_t which, const ie_complex* X_any, int64_t ldx,
                             int32_t k, ie_complex* Y_any, int64_t ldy, void* stream) {
  if (!h || !X_any || !Y_any || k < 1 || k > h->kmax || ldx < h->n || ldy < h->n ||
      (which != 0 && which != 1))
    return IE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const cplx* X;
  CKS(stage_in(h, X_any, ldx, k, h->Yb, s, &X));
  const bool ydev = is_device_ptr(Y_any);
  cplx* Y = ydev ? (cplx*)Y_any : h->Ub;
  const int64_t ldY = ydev ? ldy : h->n;
  const cplx one = make_double2(1, 0), zero = make_double2(0, 0);
  launch_spmv(h->P, which == 0 ? one : zero, which == 1 ? one : zero, X, X == h->Yb ? h->n : ldx,
              nullptr, k, Y, ldY, s);
  if (!ydev) CKS(stage_out(h, Y, ldY, k, Y_any, ldy, s));
  return check_status(h, s);
}

// ------------------------------ HSRR ------------------------------------------------------------
// Results: h->Xh (n x k Ritz vectors, unit norm), lam/e/rho on the host (QZ order).
static ie_status hsrr_dev(ie_handle h, const cplx* U, int64_t ldu, int k, cudaStream_t s,
                          std::vector<zc>& lam, std::vector<double>& e, std::vector<double>& rho) {
  const int64_t n = h->n;
  const uint64_t seed = h->opts.seed;
  launch_copy_cols(n, k, U, ldu, h->Vh, n, s);
  launch_orth_cgs2(n, k, h->Vh, n, seed, h->salt++, h->hbuf, h->scratch, h->d_flags, s);  // V
  const cplx one = make_double2(1, 0), zero = make_double2(0, 0);
  const DiaDev& P = h->pen();
  launch_spmv(P, one, zero, h->Vh, n, nullptr, k, h->AVh, n, s);                          // AV
  launch_spmv(P, zero, one, h->Vh, n, nullptr, k, h->BVh, n, s);                          // BV
  launch_spmv(P, one, to_c(-h->sig()), h->Vh, n, nullptr, k, h->Wh, n, s);               // AV - sigma BV
  launch_orth_cgs2(n, k, h->Wh, n, seed, h->salt++, h->hbuf, h->scratch, h->d_flags, s);  // W
  launch_gram(n, k, h->Wh, n, h->AVh, n, h->Ah, (cplx*)h->scratch, s);                    // W^H A V
  launch_gram(n, k, h->Wh, n, h->BVh, n, h->Bh, (cplx*)h->scratch, s);                    // W^H B V
  CK(launch_qz(k, h->Ah, h->Bh, h->Zq, h->alpha, h->betaq, h->Mq, h->status, s));
  std::vector<cplx> al(k), be(k);
  CK(cudaMemcpyAsync(al.data(), h->alpha, sizeof(cplx) * k, cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(be.data(), h->betaq, sizeof(cplx) * k, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  lam.resize(k);
  std::vector<cplx> lamc(k);
  const double inf = std::numeric_limits<double>::infinity();
  for (int i = 0; i < k; ++i) {
    const zc b = to_z(be[i]);
    lam[i] = (b == zc(0, 0)) ? zc(inf, 0) : to_z(al[i]) / b;
    lamc[i] = std::isfinite(lam[i].real()) && std::isfinite(lam[i].imag()) ? to_c(lam[i])
                                                                            : make_double2(inf, 0);
  }
  CK(cudaMemcpyAsync(h->d_lam, lamc.data(), sizeof(cplx) * k, cudaMemcpyHostToDevice, s));
  launch_gemm_small(n, k, h->Vh, n, h->Mq, h->Xh, n, s);                                  // x = V P_R V_R
  launch_normalize_cols(n, k, h->Xh, n, h->scratch, s);
  launch_residual_norms(P, k, h->Xh, n, h->d_lam, h->d_rn, h->scratch, s);
  std::vector<double> rn(3 * k);
  CK(cudaMemcpyAsync(rn.data(), h->d_rn, sizeof(double) * 3 * k, cudaMemcpyDeviceToHost, s));
  CKS(check_status(h, s));
  e.resize(k);
  rho.resize(k);
  const double scale_e = std::abs(h->ctr()) + h->radius;
  for (int i = 0; i < k; ++i) {
    const bool fin = std::isfinite(lam[i].real()) && std::isfinite(lam[i].imag());
    const double r = std::sqrt(rn[3 * i]), bx = std::sqrt(rn[3 * i + 1]), xn = std::sqrt(rn[3 * i + 2]);
    e[i] = fin ? r / (scale_e * bx) : inf;
    rho[i] = fin ? r / ((h->nA() + std::abs(lam[i]) * h->nB()) * xn) : inf;
  }
  return IE_OK;
}

extern "C" ie_status ie_hsrr(ie_handle h, const ie_complex* U_any, int64_t ldu, int32_t k,
                             ie_complex* h_lambda, ie_complex* X_any, int64_t ldx, double* h_e,
                             double* h_rho, void* stream) {
  if (!h || !U_any || k < 1 || k > h->kmax || ldu < h->n || (X_any && ldx < h->n)) return IE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const cplx* U;
  CKS(stage_in(h, U_any, ldu, k, h->Ub, s, &U));
  std::vector<zc> lam;
  std::vector<double> e, rho;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  ie_status st = hsrr_dev(h, U, U == h->Ub ? h->n : ldu, k, s, lam, e, rho);
  cudaEventRecord(e1, s);
  cudaStreamSynchronize(s);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->stats.t_hsrr_ms = ms;
  if (st != IE_OK) return st;
  for (int i = 0; i < k; ++i) {
    if (h_lambda) { h_lambda[i].re = lam[i].real(); h_lambda[i].im = lam[i].imag(); }
    if (h_e) h_e[i] = e[i];
    if (h_rho) h_rho[i] = rho[i];
  }
  if (X_any) CKS(stage_out(h, h->Xh, h->n, k, X_any, ldx, s));
  return check_status(h, s);
}

// ------------------------------ drivers ----------------------------------------------------------
// IE_SOLVE_LOG=1: one line per outer iteration of the drivers on stderr
static bool solve_log() {
  static const bool on = [] {
    const char* v = getenv("IE_SOLVE_LOG");
    return v && v[0] == '1';
  }();
  return on;
}

static bool in_disk(ie_handle h, zc l) {
  return std::isfinite(l.real()) && std::isfinite(l.imag()) && std::abs(l - h->ctr()) < h->radius;
}

// Alg. 1 / Alg. 2 on the handle's current side (the pencil (A, B), or its adjoint).
static ie_status solve_driver(ie_handle h, const ie_complex* Y0_any, int64_t ldy0,
                              ie_complex* h_lambda, ie_complex* X_any, int64_t ldx, double* h_rho,
                              double* h_e, int32_t* n_found, ie_stats* stats, cudaStream_t s) {
  const int k = h->kmax;
  const int64_t n = h->n;
  // starting block
  if (Y0_any) {
    if (is_device_ptr(Y0_any)) {
      launch_copy_cols(n, k, (const cplx*)Y0_any, ldy0, h->Yb, n, s);
    } else {
      CK(cudaMemcpy2DAsync(h->Yb, sizeof(cplx) * n, Y0_any, sizeof(cplx) * ldy0, sizeof(cplx) * n,
                           k, cudaMemcpyHostToDevice, s));
    }
  } else {
    launch_random_block(n, k, h->Yb, n, h->opts.seed, 0xA5A5u, s);
    launch_orth_cgs2(n, k, h->Yb, n, h->opts.seed, 0x5A5Au, h->hbuf, h->scratch, h->d_flags, s);
  }
  h->salt = 1;
  ie_stats& S = h->stats;
  const double t_factor = S.t_factor_ms;
  S = ie_stats{};
  S.t_factor_ms = t_factor;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  std::vector<zc> lam;
  std::vector<double> e, rho;
  std::vector<char> filt;
  int prev = -1, nf = 0;
  bool converged = false, any_noconv = false;
  int pc = h->p;
  ie_status st = IE_OK;
  for (int t = 1; t <= h->opts.max_outer; ++t) {
    cudaEventRecord(e0, s);
    bool nc = false;
    if (h->opts.driver == 1) {
      st = filter_dev(h, h->Yb, n, k, h->Ub, n, h->p, false, s, &nc);       // Alg. 1 filter step
    } else {
      st = filter_dev(h, h->Yb, n, k, h->Ub, n, pc, t > 1, s, &nc);         // Alg. 2 filter step
    }
    cudaEventRecord(e1, s);
    if (st != IE_OK) break;
    cudaStreamSynchronize(s);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    S.t_filter_ms += ms;
    any_noconv |= nc;
    cudaEventRecord(e0, s);
    st = hsrr_dev(h, h->Ub, n, k, s, lam, e, rho);                           // extraction step
    cudaEventRecord(e1, s);
    if (st != IE_OK) break;
    cudaStreamSynchronize(s);
    cudaEventElapsedTime(&ms, e0, e1);
    S.t_hsrr_ms += ms;
    // ghost filter and stop test (Sec. 3.2)
    filt.assign(k, 0);
    nf = 0;
    bool all_conv = true;
    double mr = 0.0;
    for (int i = 0; i < k; ++i) {
      filt[i] = in_disk(h, lam[i]) && e[i] < h->opts.tau_g;
      if (filt[i]) {
        ++nf;
        mr = std::max(mr, rho[i]);
        if (!(rho[i] < h->opts.tau)) all_conv = false;
      }
    }
    if (solve_log()) {
      int unconv = 0, inside = 0;
      double emax = 0.0;
      for (int i = 0; i < k; ++i) {
        if (filt[i] && !(rho[i] < h->opts.tau)) ++unconv;
        if (in_disk(h, lam[i])) ++inside;
        if (filt[i]) emax = std::max(emax, e[i]);
      }
      fprintf(stderr, "ie_solve%s t=%d p=%d: Ritz values in D %d, filtered %d, not yet converged %d, "
              "max rho %.3e, max e %.3e, gmres steps %d..%d\n", h->side ? " (adjoint)" : "", t,
              pc, inside, nf, unconv, mr, emax, h->stats.gmres_iters_min, h->stats.gmres_iters_max);
    }
    S.outer_iters = t;
    S.n_found = nf;
    S.max_rho_found = mr;
    if ((t == 1 && nf >= 1 && all_conv) || (t >= 2 && nf == prev && all_conv)) {
      converged = true;
      break;
    }
    prev = nf;
    if (h->opts.driver == 1) {
      launch_copy_cols(n, k, h->Xh, n, h->Yb, n, s);                         // Y <- Ritz vectors
    } else {
      pc *= 2;                                                               // doubling step
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != IE_OK) return st;
  // order: filtered first, each group by |lambda - c|
  std::vector<int> ord(k);
  std::iota(ord.begin(), ord.end(), 0);
  auto dist = [&](int i) {
    return (std::isfinite(lam[i].real()) && std::isfinite(lam[i].imag()))
               ? std::abs(lam[i] - h->ctr())
               : std::numeric_limits<double>::infinity();
  };
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
    if (filt[a] != filt[b]) return filt[a] > filt[b];
    return dist(a) < dist(b);
  });
  CK(cudaMemcpyAsync(h->d_perm, ord.data(), sizeof(int) * k, cudaMemcpyHostToDevice, s));
  const bool xdev = is_device_ptr(X_any);
  cplx* Xo = xdev ? (cplx*)X_any : h->Ub;
  const int64_t ldXo = xdev ? ldx : n;
  launch_permute_cols(n, k, h->Xh, n, h->d_perm, Xo, ldXo, s);
  if (!xdev) CKS(stage_out(h, Xo, ldXo, k, X_any, ldx, s));
  CKS(check_status(h, s));
  for (int i = 0; i < k; ++i) {
    const zc l = lam[ord[i]];
    h_lambda[i].re = l.real();
    h_lambda[i].im = l.imag();
    if (h_rho) h_rho[i] = rho[ord[i]];
    if (h_e) h_e[i] = e[ord[i]];
  }
  *n_found = nf;
  S.converged = converged ? 1 : 0;
  fill_solve_stats(h, &S);
  if (stats) *stats = S;
  (void)any_noconv;
  return converged ? IE_OK : IE_ERR_NOCONV;
}

extern "C" ie_status ie_solve(ie_handle h, const ie_complex* Y0_any, int64_t ldy0,
                              ie_complex* h_lambda, ie_complex* X_any, int64_t ldx, double* h_rho,
                              double* h_e, int32_t* n_found, ie_stats* stats, void* stream) {
  if (!h || !h_lambda || !X_any || !n_found || ldx < h->n) return IE_ERR_ARG;
  if (Y0_any && ldy0 < h->n) return IE_ERR_ARG;
  h->side = 0;
  return solve_driver(h, Y0_any, ldy0, h_lambda, X_any, ldx, h_rho, h_e, n_found, stats,
                      (cudaStream_t)stream);
}

// ------------------------------ batched solves ---------------------------------------------------
// A pool of host threads, each running whole drivers of the items it takes; item work goes to
// one stream per item, so kernels and host round trips of different problems overlap.
extern "C" ie_status ie_solve_batch(ie_batch_item* items, int32_t nb, int32_t max_workers) {
  if (!items || nb < 1) return IE_ERR_ARG;
  std::set<ie_handle> seen;
  for (int i = 0; i < nb; ++i) {
    const ie_batch_item& it = items[i];
    if (!it.h || !it.h_lambda || !it.X_any || it.ldx < it.h->n) return IE_ERR_ARG;
    if (it.Y0_any && it.ldy0 < it.h->n) return IE_ERR_ARG;
    if (!seen.insert(it.h).second) return IE_ERR_ARG;
  }
  int workers = max_workers > 0 ? max_workers : std::min(nb, 16);
  workers = std::min(workers, (int)nb);
  std::atomic<int> next{0};
  auto work = [&]() {
    for (int i = next.fetch_add(1); i < nb; i = next.fetch_add(1)) {
      ie_batch_item& it = items[i];
      ie_handle h = it.h;
      if (cudaSetDevice(h->dev) != cudaSuccess) { it.status = IE_ERR_CUDA; continue; }
      cudaStream_t s = (cudaStream_t)it.stream;
      bool own = false;
      if (!s) {
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
          it.status = IE_ERR_CUDA;
          continue;
        }
        own = true;
      }
      h->side = 0;
      int32_t nf = 0;
      ie_stats st{};
      it.status = solve_driver(h, it.Y0_any, it.ldy0, it.h_lambda, it.X_any, it.ldx, it.h_rho,
                               it.h_e, &nf, &st, s);
      it.n_found = nf;
      it.stats = st;
      if (own) {
        cudaStreamSynchronize(s);
        cudaStreamDestroy(s);
      }
    }
  };
  if (workers == 1) {
    work();
  } else {
    std::vector<std::thread> pool;
    pool.reserve(workers);
    for (int w = 0; w < workers; ++w) pool.emplace_back(work);
    for (auto& t : pool) t.join();
  }
  for (int i = 0; i < nb; ++i)
    if (items[i].status != IE_OK) return (ie_status)items[i].status;
  return IE_OK;
}

// ------------------------------ fused batch ----------------------------------------------------
// All problems of a batch advance together: every Arnoldi step applies G to the active columns
// of every problem with ONE band-solve launch per element type (band_solve_batch_kernel), the
// per-problem Krylov kernels follow on the same stream, and one synchronisation serves all
// problems' convergence tests. A problem whose filter is complete runs its HSRR and stop test,
// then either finishes or starts its next outer iteration while the others keep stepping.
namespace {
struct GReq {
  ie_handle h;
  const cplx* V;
  int64_t ldv;
  const int64_t* d_off;
  int k;
  cplx* GV;
  int64_t ldg;
};

// pinned host scratch, reused across calls of one fused solve
struct Pinned {
  void* p = nullptr;
  size_t cap = 0;
  ~Pinned() { if (p) cudaFreeHost(p); }
  void* get(size_t bytes) {
    if (bytes > cap) {
      if (p) cudaFreeHost(p);
      p = nullptr;
      cap = 0;
      if (cudaMallocHost(&p, bytes) != cudaSuccess) return nullptr;
      cap = bytes;
    }
    return p;
  }
};
}  // namespace

// G applied to every request (Eq. linearsolve2), one batched band-solve launch per element type
// (complex128, complex64); mixed-precision requests refine in lockstep, each until its own
// target (as apply_G_mixed), with one synchronisation per refinement step for all of them.
static ie_status apply_G_batch(std::vector<GReq>& reqs, BandSolveBatch* bb, Pinned& pin,
                               cudaStream_t s) {
  if (reqs.empty()) return IE_OK;
  band_solve_batch_clear(bb);
  std::vector<size_t> mixed;
  for (size_t r = 0; r < reqs.size(); ++r) {
    GReq& g = reqs[r];
    ie_handle h = g.h;
    launch_spmv(h->pen(), make_double2(0, 0), make_double2(1, 0), g.V, g.ldv, g.d_off, g.k,
                h->BVw, h->n, s);
    const int64_t ps = h->n * (int64_t)h->kmax;
    if (h->precision == 0) {
      band_solve_batch_add64(bb, h->q, h->n, h->kl, h->n_pad, h->L64, h->U64, h->piv, h->dinv,
                             h->Tb, h->Hb, h->Uinvb, h->d_weights, h->BVw, h->n, g.k, h->Xp,
                             h->n, ps, h->status);
    } else {
      launch_to_c64(h->n, g.k, h->BVw, h->n, h->BV32, h->n, s);
      band_solve_batch_add32(bb, h->q, h->n, h->kl, h->n_pad, h->L32, h->klp, h->U32, h->kv,
                             h->piv, h->dinv32, h->T32, h->Hb, h->Ub32, h->d_weights, h->BV32,
                             h->n, 0, g.k, h->Y32, h->n, ps, h->Xp, h->n, ps, 0, h->status);
      mixed.push_back(r);
    }
  }
  CK(band_solve_batch_launch(bb, s));
  // lockstep FP64 refinement of the mixed-precision requests (see apply_G_mixed)
  struct Ref { size_t r; double prev, last; bool on; };
  std::vector<Ref> ref;
  for (size_t r : mixed) {
    ie_handle h = reqs[r].h;
    const bool skip = h->ref_eps0 > 0.0 && 10.0 * h->ref_eps0 <= h->refine_target;
    ref.push_back({r, -1.0, 0.0, !skip && h->refine > 0});
  }
  for (int it = 1;; ++it) {
    bool any = false;
    band_solve_batch_clear(bb);
    size_t off = 0;
    std::vector<size_t> offs(ref.size(), 0);
    for (size_t i = 0; i < ref.size(); ++i) {
      Ref& f = ref[i];
      ie_handle h = reqs[f.r].h;
      if (!f.on || it > h->refine) { f.on = false; continue; }
      any = true;
      const int k = reqs[f.r].k;
      const int64_t n = h->n, ps = n * (int64_t)h->kmax;
      launch_pole_residual(h->pen(), h->d_poles, h->q, k, h->BVw, n, h->Xp, n, ps, h->R32, n,
                           ps, s);
      band_solve_batch_add32(bb, h->q, n, h->kl, h->n_pad, h->L32, h->klp, h->U32, h->kv, h->piv,
                             h->dinv32, h->T32, h->Hb, h->Ub32, h->d_weights, h->R32, n, ps, k,
                             h->Y32, n, ps, h->Xp, n, ps, 1, h->status);
      offs[i] = off;
      off += (size_t)h->q * k * 2;
    }
    if (!any) break;
    CK(band_solve_batch_launch(bb, s));
    unsigned* hn = (unsigned*)pin.get(off * sizeof(unsigned));
    if (!hn) return IE_ERR_OOM;
    for (size_t i = 0; i < ref.size(); ++i) {
      Ref& f = ref[i];
      if (!f.on) continue;
      ie_handle h = reqs[f.r].h;
      const int k = reqs[f.r].k;
      const int64_t n = h->n, ps = n * (int64_t)h->kmax;
      const size_t nn2 = (size_t)h->q * k * 2;
      CK(cudaMemsetAsync(h->d_rnrm, 0, sizeof(unsigned) * nn2, s));
      launch_refine_add(h->q, n, k, h->Y32, n, ps, h->Xp, n, ps, h->d_rnrm, s);
      CK(cudaMemcpyAsync(hn + offs[i], h->d_rnrm, sizeof(unsigned) * nn2, cudaMemcpyDeviceToHost, s));
    }
    CK(cudaStreamSynchronize(s));
    for (size_t i = 0; i < ref.size(); ++i) {
      Ref& f = ref[i];
      if (!f.on) continue;
      ie_handle h = reqs[f.r].h;
      const size_t nn2 = (size_t)h->q * reqs[f.r].k * 2;
      h->refine_solves += 1;
      double d = 0.0;
      for (size_t e = 0; e < nn2; e += 2) {
        float dm, xm;
        std::memcpy(&dm, &hn[offs[i] + e], sizeof(float));
        std::memcpy(&xm, &hn[offs[i] + e + 1], sizeof(float));
        if (xm > 0.0f) d = std::max(d, (double)dm / (double)xm);
      }
      f.last = d;
      if (it == 1) h->ref_eps0 = d;
      if (f.prev > 0.0) {
        if (d > 0.5 * f.prev) { f.on = false; continue; }
        h->ref_c = std::min(1.0, d / f.prev);
      }
      const double c = f.prev > 0.0 ? d / f.prev : (h->ref_c > 0.0 ? 10.0 * h->ref_c : 1.0);
      if (d * std::min(1.0, c) <= h->refine_target) f.on = false;
      f.prev = d;
    }
  }
  for (auto& f : ref) reqs[f.r].h->refine_last_corr = f.last;
  for (GReq& g : reqs) {
    ie_handle h = g.h;
    const int64_t ps = h->n * (int64_t)h->kmax;
    if (h->precision == 0)
      launch_pole_sum(h->q, h->n, g.k, h->Xp, h->n, ps, g.GV, g.ldg, s);
    else
      launch_pole_wsum(h->q, h->n, g.k, h->Xp, h->n, ps, h->d_weights, g.GV, g.ldg, s);
    h->g_columns += g.k;
  }
  return IE_OK;
}

extern "C" ie_status ie_solve_batch_fused(ie_batch_item* items, int32_t nb, void* stream) {
  if (!items || nb < 1) return IE_ERR_ARG;
  std::set<ie_handle> seen;
  int dev = -1;
  cudaGetDevice(&dev);
  for (int i = 0; i < nb; ++i) {
    const ie_batch_item& it = items[i];
    if (!it.h || !it.h_lambda || !it.X_any || it.ldx < it.h->n) return IE_ERR_ARG;
    if (it.Y0_any && it.ldy0 < it.h->n) return IE_ERR_ARG;
    if (!seen.insert(it.h).second || it.h->dev != dev) return IE_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  BandSolveBatch* bb = band_solve_batch_create();
  Pinned pin, pin2;
  struct FItem {
    ie_batch_item* it;
    ie_handle h;
    int phase = 0;   // 0: start a filter, 1: Arnoldi steps, 2: filter done, 3: finished
    int t = 1, pc = 0, prev = -1, nf = 0, nshift = 0;
    bool converged = false, reuse = false, noconv = false;
    double rmax = 1.0, odd = 0.0;
    std::vector<int> act;
    std::vector<zc> lam;
    std::vector<double> e, rho;
    std::vector<char> filt;
  };
  std::vector<FItem> F(nb);
  ie_status first_bad = IE_OK;
  auto fail = [&](FItem& f, ie_status st) {
    f.it->status = st;
    f.phase = 3;
    if (first_bad == IE_OK) first_bad = st;
  };
  for (int i = 0; i < nb; ++i) {
    FItem& f = F[i];
    f.it = &items[i];
    f.h = items[i].h;
    ie_handle h = f.h;
    h->side = 0;
    f.pc = h->p;
    f.it->status = IE_OK;
    f.it->n_found = 0;
    const int k = h->kmax;
    const int64_t n = h->n;
    if (f.it->Y0_any) {
      if (is_device_ptr(f.it->Y0_any))
        launch_copy_cols(n, k, (const cplx*)f.it->Y0_any, f.it->ldy0, h->Yb, n, s);
      else if (cudaMemcpy2DAsync(h->Yb, sizeof(cplx) * n, f.it->Y0_any, sizeof(cplx) * f.it->ldy0,
                                 sizeof(cplx) * n, k, cudaMemcpyHostToDevice, s) != cudaSuccess) {
        fail(f, IE_ERR_CUDA);
        continue;
      }
    } else {
      launch_random_block(n, k, h->Yb, n, h->opts.seed, 0xA5A5u, s);
      launch_orth_cgs2(n, k, h->Yb, n, h->opts.seed, 0x5A5Au, h->hbuf, h->scratch, h->d_flags, s);
    }
    h->salt = 1;
    const double t_factor = h->stats.t_factor_ms;
    h->stats = ie_stats{};
    h->stats.t_factor_ms = t_factor;
  }
  while (true) {
    // ---- requests of this step
    std::vector<GReq> reqs;
    std::vector<int> starting, stepping;
    size_t nres = 0;
    for (int i = 0; i < nb; ++i) {
      FItem& f = F[i];
      ie_handle h = f.h;
      if (f.phase == 0) {
        const int k = h->kmax;
        f.reuse = h->opts.driver == 2 && f.t > 1;
        std::vector<zc> sh, cw;
        outer_coeffs(f.pc, sh, cw, f.odd);
        f.nshift = (int)sh.size();
        if (ensure_shift_capacity(h, std::max(f.nshift, 1)) != IE_OK) { fail(f, IE_ERR_OOM); continue; }
        std::vector<cplx> a(f.nshift), b(f.nshift);
        for (int j = 0; j < f.nshift; ++j) { a[j] = to_c(sh[j]); b[j] = to_c(cw[j]); }
        if (f.nshift) {
          cudaMemcpyAsync(h->d_shifts, a.data(), sizeof(cplx) * f.nshift, cudaMemcpyHostToDevice, s);
          cudaMemcpyAsync(h->d_cw, b.data(), sizeof(cplx) * f.nshift, cudaMemcpyHostToDevice, s);
        }
        f.noconv = false;
        f.rmax = 1.0;
        if (!f.reuse) {
          h->refine_target = kRefineFull;
          reqs.push_back({h, h->Yb, h->n, nullptr, k, h->Wb, h->n});   // Ytilde = G(Y)
          starting.push_back(i);
        } else {
          // Alg. 2: the kept Krylov spaces, every shift of the doubled set re-solved
          f.act.clear();
          for (int c = 0; c < k; ++c) {
            h->conv_h[c] = (h->beta_h[c] > 0.0 && f.nshift > 0) ? 0 : 1;
            if (!h->conv_h[c] && h->jc_h[c] > 0) f.act.push_back(c);
          }
          if (!f.act.empty()) {
            cudaMemcpyAsync(h->d_act, f.act.data(), sizeof(int) * f.act.size(),
                            cudaMemcpyHostToDevice, s);
            launch_givens(h->K, h->d_act, (int)f.act.size(), h->d_shifts, f.nshift, h->rot_c,
                          h->rot_s, h->gvec, 1, h->d_res, s);
            stepping.push_back(i);
            nres += f.act.size();
          }
          f.phase = 1;
        }
      } else if (f.phase == 1) {
        f.act.clear();
        for (int c = 0; c < h->kmax; ++c)
          if (!h->conv_h[c]) {
            if (h->jc_h[c] >= h->m_max) { f.noconv = true; continue; }
            f.act.push_back(c);
          }
        if (f.act.empty()) { f.phase = 2; continue; }
        const int kact = (int)f.act.size();
        cudaMemcpyAsync(h->d_act, f.act.data(), sizeof(int) * kact, cudaMemcpyHostToDevice, s);
        launch_active_offsets(h->K, h->d_act, kact, h->d_off, s);
        if (h->precision == 1) h->refine_target = std::min(1e-2, h->opts.gmres_tol / (50.0 * f.rmax));
        reqs.push_back({h, h->K.V, h->n, h->d_off, kact, h->Wb, h->n});
        stepping.push_back(-1 - i);   // marks an Arnoldi step (decoded below)
        nres += kact;
      }
    }
    if (!reqs.empty()) {
      const ie_status gs = apply_G_batch(reqs, bb, pin2, s);
      if (gs != IE_OK) {
        for (auto& f : F) if (f.phase < 3) fail(f, gs);
        break;
      }
    }
    for (GReq& g : reqs) g.h->refine_target = kRefineFull;
    // ---- Krylov work of this step and one read-back for all problems
    size_t nbeta = 0;
    for (int i : starting) nbeta += F[i].h->kmax;
    double* hb = (double*)pin.get(sizeof(double) * (nres + nbeta + 1));
    if (!hb) { for (auto& f : F) if (f.phase < 3) fail(f, IE_ERR_OOM); break; }
    size_t off = 0;
    std::vector<size_t> boff(nb, 0), roff(nb, 0);
    for (int i : starting) {
      ie_handle h = F[i].h;
      launch_krylov_start(h->K, h->kmax, h->Wb, h->n, h->scratch, s);
      boff[i] = off;
      cudaMemcpyAsync(hb + off, h->K.beta, sizeof(double) * h->kmax, cudaMemcpyDeviceToHost, s);
      off += h->kmax;
    }
    for (int code : stepping) {
      const bool arnoldi = code < 0;
      const int i = arnoldi ? -1 - code : code;
      FItem& f = F[i];
      ie_handle h = f.h;
      const int kact = (int)f.act.size();
      if (arnoldi) {
        launch_arnoldi_cgs2(h->K, h->d_act, kact, h->Wb, h->n, h->hbuf, h->scratch, s);
        launch_givens(h->K, h->d_act, kact, h->d_shifts, f.nshift, h->rot_c, h->rot_s, h->gvec, 0,
                      h->d_res, s);
      }
      roff[i] = off;
      cudaMemcpyAsync(hb + off, h->d_res, sizeof(double) * kact, cudaMemcpyDeviceToHost, s);
      off += kact;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) {
      for (auto& f : F) if (f.phase < 3) fail(f, IE_ERR_CUDA);
      break;
    }
    for (int i = 0; i < nb; ++i) flush_solve_timing(F[i].h);
    for (int i : starting) {
      FItem& f = F[i];
      ie_handle h = f.h;
      const int k = h->kmax;
      for (int c = 0; c < k; ++c) {
        h->beta_h[c] = hb[boff[i] + c];
        h->jc_h[c] = 0;
        h->conv_h[c] = (h->beta_h[c] > 0.0 && f.nshift > 0) ? 0 : 1;
      }
      f.phase = 1;
    }
    for (int code : stepping) {
      const bool arnoldi = code < 0;
      const int i = arnoldi ? -1 - code : code;
      FItem& f = F[i];
      ie_handle h = f.h;
      double rm = 0.0;
      for (size_t a = 0; a < f.act.size(); ++a) {
        const int c = f.act[a];
        const double r = hb[roff[i] + a];
        if (arnoldi) h->jc_h[c] += 1;
        if (r <= h->opts.gmres_tol) h->conv_h[c] = 1;
        else rm = std::max(rm, r);
      }
      f.rmax = rm > 0.0 ? rm : 1.0;
    }
    // ---- problems whose filter is complete: combine, HSRR, stop test (Sec. 3.2)
    for (int i = 0; i < nb; ++i) {
      FItem& f = F[i];
      if (f.phase != 2) continue;
      ie_handle h = f.h;
      const int k = h->kmax;
      const int64_t n = h->n;
      launch_krylov_combine(h->K, k, h->d_shifts, h->d_cw, f.nshift, f.odd, h->Rscr, h->zbuf, h->Ub,
                            n, s);
      int mx = 0, mn = 1 << 30;
      for (int c = 0; c < k; ++c) { mx = std::max(mx, h->jc_h[c]); mn = std::min(mn, h->jc_h[c]); }
      h->stats.gmres_iters_max = mx;
      h->stats.gmres_iters_min = mn;
      h->stats.p_final = f.pc;
      const ie_status hs = hsrr_dev(h, h->Ub, n, k, s, f.lam, f.e, f.rho);
      if (hs != IE_OK) { fail(f, hs); continue; }
      f.filt.assign(k, 0);
      int nf = 0;
      bool all_conv = true;
      double mr = 0.0;
      for (int j = 0; j < k; ++j) {
        f.filt[j] = in_disk(h, f.lam[j]) && f.e[j] < h->opts.tau_g;
        if (f.filt[j]) {
          ++nf;
          mr = std::max(mr, f.rho[j]);
          if (!(f.rho[j] < h->opts.tau)) all_conv = false;
        }
      }
      f.nf = nf;
      h->stats.outer_iters = f.t;
      h->stats.n_found = nf;
      h->stats.max_rho_found = mr;
      if ((f.t == 1 && nf >= 1 && all_conv) || (f.t >= 2 && nf == f.prev && all_conv)) {
        f.converged = true;
      } else if (f.t >= h->opts.max_outer) {
        f.converged = false;
      } else {
        f.prev = nf;
        if (h->opts.driver == 1) launch_copy_cols(n, k, h->Xh, n, h->Yb, n, s);   // Y <- Ritz vectors
        else f.pc *= 2;                                                             // doubling step
        f.t += 1;
        f.phase = 0;
        continue;
      }
      // outputs: filtered pairs first, each group by |lambda - c| (as ie_solve)
      std::vector<int> ord(k);
      std::iota(ord.begin(), ord.end(), 0);
      auto dist = [&](int j) {
        return (std::isfinite(f.lam[j].real()) && std::isfinite(f.lam[j].imag()))
                   ? std::abs(f.lam[j] - h->ctr())
                   : std::numeric_limits<double>::infinity();
      };
      std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
        if (f.filt[a] != f.filt[b]) return f.filt[a] > f.filt[b];
        return dist(a) < dist(b);
      });
      cudaMemcpyAsync(h->d_perm, ord.data(), sizeof(int) * k, cudaMemcpyHostToDevice, s);
      const bool xdev = is_device_ptr(f.it->X_any);
      cplx* Xo = xdev ? (cplx*)f.it->X_any : h->Ub;
      const int64_t ldXo = xdev ? f.it->ldx : n;
      launch_permute_cols(n, k, h->Xh, n, h->d_perm, Xo, ldXo, s);
      if (!xdev && stage_out(h, Xo, ldXo, k, f.it->X_any, f.it->ldx, s) != IE_OK) {
        fail(f, IE_ERR_CUDA);
        continue;
      }
      const ie_status cs = check_status(h, s);
      if (cs != IE_OK) { fail(f, cs); continue; }
      for (int j = 0; j < k; ++j) {
        const zc l = f.lam[ord[j]];
        f.it->h_lambda[j].re = l.real();
        f.it->h_lambda[j].im = l.imag();
        if (f.it->h_rho) f.it->h_rho[j] = f.rho[ord[j]];
        if (f.it->h_e) f.it->h_e[j] = f.e[ord[j]];
      }
      f.it->n_found = nf;
      h->stats.converged = f.converged ? 1 : 0;
      fill_solve_stats(h, &h->stats);
      f.it->stats = h->stats;
      f.it->status = f.converged ? IE_OK : IE_ERR_NOCONV;
      if (!f.converged && first_bad == IE_OK) first_bad = IE_ERR_NOCONV;
      f.phase = 3;
    }
    bool all_done = true;
    for (auto& f : F) all_done &= f.phase == 3;
    if (all_done) break;
  }
  band_solve_batch_destroy(bb);
  for (int i = 0; i < nb; ++i)
    if (items[i].status != IE_OK) return (ie_status)items[i].status;
  return first_bad;
}

// ------------------------------ adjoint pencil --------------------------------------------------
namespace {
struct SideGuard {   // the adjoint side for the guard's lifetime
  ie_handle h;
  explicit SideGuard(ie_handle h_) : h(h_) { h->side = 1; }
  ~SideGuard() { h->side = 0; }
};
}  // namespace

extern "C" ie_status ie_apply_GH(ie_handle h, const ie_complex* V_any, int64_t ldv, int32_t k,
                                 ie_complex* GV_any, int64_t ldgv, void* stream) {
  if (!h || !h->adj || !V_any || !GV_any || k < 1 || k > h->kmax || ldv < h->n || ldgv < h->n)
    return IE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  SideGuard g(h);
  const cplx* V;
  CKS(stage_in(h, V_any, ldv, k, h->Yb, s, &V));
  const bool gdev = is_device_ptr(GV_any);
  cplx* G = gdev ? (cplx*)GV_any : h->Ub;
  const int64_t ldG = gdev ? ldgv : h->n;
  CKS(apply_G_dev(h, V, V == h->Yb ? h->n : ldv, nullptr, k, G, ldG, s));
  if (!gdev) CKS(stage_out(h, G, ldG, k, GV_any, ldgv, s));
  h->stats.g_columns = h->g_columns;
  return check_status(h, s);
}

extern "C" ie_status ie_solve_left(ie_handle h, const ie_complex* h_lambda, int32_t nl,
                                   const ie_complex* Y0_any, int64_t ldy0, ie_complex* Y_any,
                                   int64_t ldy, ie_complex* h_lambda_left, double* h_rho_left,
                                   ie_stats* stats, void* stream) {
  if (!h || !h->adj || !h_lambda || !Y_any || nl < 1 || nl > h->kmax || ldy < h->n) return IE_ERR_ARG;
  if (Y0_any && ldy0 < h->n) return IE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int k = h->kmax;
  const int64_t n = h->n;
  std::vector<ie_complex> mu(k);
  std::vector<double> rho(k);
  int32_t nf = 0;
  ie_status st;
  {
    SideGuard g(h);
    // the driver leaves its ordered Ritz vectors in h->Wb (n x k)
    st = solve_driver(h, Y0_any, ldy0, mu.data(), (ie_complex*)h->Wb, n, rho.data(), nullptr, &nf,
                      stats, s);
  }
  if (st != IE_OK && st != IE_ERR_NOCONV) return st;
  // pair each requested eigenvalue with the nearest conj(mu_j), one-to-one
  std::vector<int> perm(nl, 0);
  std::vector<char> used(k, 0);
  bool paired = true;
  for (int i = 0; i < nl; ++i) {
    const zc li = to_z(h_lambda[i]);
    int best = -1;
    double bd = std::numeric_limits<double>::infinity();
    for (int j = 0; j < k; ++j) {
      const zc mj = std::conj(to_z(mu[j]));
      if (!std::isfinite(mj.real()) || !std::isfinite(mj.imag())) continue;
      const double d = std::abs(mj - li);
      if (d < bd) { bd = d; best = j; }
    }
    if (best < 0) { paired = false; continue; }
    if (used[best] || !(bd <= 1e-8 * std::max(std::abs(li), h->radius))) paired = false;
    used[best] = 1;
    perm[i] = best;
    if (h_lambda_left) {
      h_lambda_left[i].re = mu[best].re;
      h_lambda_left[i].im = -mu[best].im;
    }
    if (h_rho_left) h_rho_left[i] = rho[best];
  }
  CK(cudaMemcpyAsync(h->d_perm, perm.data(), sizeof(int) * nl, cudaMemcpyHostToDevice, s));
  const bool ydev = is_device_ptr(Y_any);
  cplx* Yo = ydev ? (cplx*)Y_any : h->Ub;
  const int64_t ldYo = ydev ? ldy : n;
  launch_permute_cols(n, nl, h->Wb, n, h->d_perm, Yo, ldYo, s);
  if (!ydev) CKS(stage_out(h, Yo, ldYo, nl, Y_any, ldy, s));
  CKS(check_status(h, s));
  if (stats) fill_solve_stats(h, stats);
  if (st != IE_OK || !paired) return IE_ERR_NOCONV;
  return IE_OK;
}

extern "C" ie_status ie_eig_sensitivity(ie_handle h, const ie_complex* X_any, int64_t ldx,
                                        const ie_complex* Y_any, int64_t ldy, int32_t nf,
                                        ie_complex alpha, ie_complex* S_any, int64_t lds,
                                        const ie_complex* h_gbar, double* grad_any, void* stream) {
  if (!h || !X_any || !Y_any || nf < 1 || nf > h->kmax || ldx < h->n || ldy < h->n) return IE_ERR_ARG;
  if ((S_any && lds < h->n) || (grad_any && !h_gbar)) return IE_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = h->n;
  const cplx* X;
  const cplx* Y;
  CKS(stage_in(h, X_any, ldx, nf, h->Yb, s, &X));
  CKS(stage_in(h, Y_any, ldy, nf, h->Ub, s, &Y));
  const int64_t ldX = (X == h->Yb) ? n : ldx, ldY = (Y == h->Ub) ? n : ldy;
  const bool sdev = S_any && is_device_ptr(S_any);
  cplx* S = S_any ? (sdev ? (cplx*)S_any : h->Xh) : nullptr;
  const int64_t ldS = sdev ? lds : n;
  double* grad = nullptr;
  cplx* gb = nullptr;
  if (grad_any) {
    if (is_device_ptr(grad_any)) {
      grad = grad_any;
    } else {
      if (!h->d_grad) CK(h->alloc(&h->d_grad, (size_t)n));
      grad = h->d_grad;
    }
    std::vector<cplx> g(nf);
    for (int i = 0; i < nf; ++i) g[i] = make_double2(h_gbar[i].re, h_gbar[i].im);
    CK(cudaMemcpyAsync(h->betaq, g.data(), sizeof(cplx) * nf, cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));
    gb = h->betaq;
  }
  launch_sensitivity(h->P, nf, X, ldX, Y, ldY, make_double2(alpha.re, alpha.im), h->Wb, h->alpha,
                     S, ldS, gb, grad, s);
  if (S_any && !sdev) CKS(stage_out(h, S, ldS, nf, S_any, lds, s));
  if (grad_any && grad != grad_any)
    CK(cudaMemcpyAsync(grad_any, grad, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
  return check_status(h, s);
}

// ------------------------------ introspection -----------------------------------------------
extern "C" ie_status ie_get_coeffs(ie_handle h, ie_complex* h_poles, ie_complex* h_weights,
                                   ie_complex* h_shifts, ie_complex* h_cweights, int32_t* n_shift,
                                   double* odd_coef) {
  if (!h) return IE_ERR_ARG;
  for (int i = 0; i < h->q; ++i) {
    if (h_poles) { h_poles[i].re = h->poles[i].real(); h_poles[i].im = h->poles[i].imag(); }
    if (h_weights) { h_weights[i].re = h->weights[i].real(); h_weights[i].im = h->weights[i].imag(); }
  }
  std::vector<zc> sh, cw;
  double odd = 0;
  outer_coeffs(h->p, sh, cw, odd);
  for (size_t j = 0; j < sh.size(); ++j) {
    if (h_shifts) { h_shifts[j].re = sh[j].real(); h_shifts[j].im = sh[j].imag(); }
    if (h_cweights) { h_cweights[j].re = cw[j].real(); h_cweights[j].im = cw[j].imag(); }
  }
  if (n_shift) *n_shift = (int32_t)sh.size();
  if (odd_coef) *odd_coef = odd;
  return IE_OK;
}

extern "C" ie_status ie_get_factor(ie_handle h, int32_t pole, ie_complex* h_ab, int32_t* h_ipiv,
                                   int32_t* kl, int32_t* ldab) {
  if (!h || pole < 0 || pole >= h->q || (!h->AB && !h->L32)) return IE_ERR_ARG;
  if (kl) *kl = h->kl;
  if (ldab) *ldab = h->ldab;
  if (h_ab && h->AB) {
    CK(cudaMemcpy(h_ab, h->AB + (int64_t)pole * h->n_pad * h->ldab,
                  sizeof(cplx) * (size_t)h->n * h->ldab, cudaMemcpyDeviceToHost));
  } else if (h_ab) {
    // complex64 factors, widened exactly: L from L32, U above the diagonal from U32, U(j,j)
    const int64_t n = h->n, np = h->n_pad;
    const int k_l = h->kl, kv = h->kv, ld = h->ldab, klp = h->klp;
    std::vector<float2> L((size_t)np * klp), U((size_t)np * kv), D((size_t)np);
    CK(cudaMemcpy(L.data(), h->L32 + (int64_t)pole * np * klp, sizeof(float2) * L.size(),
                  cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(U.data(), h->U32 + (int64_t)pole * np * kv, sizeof(float2) * U.size(),
                  cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(D.data(), h->diag32 + (int64_t)pole * np, sizeof(float2) * D.size(),
                  cudaMemcpyDeviceToHost));
    for (int64_t j = 0; j < n; ++j) {
      ie_complex* col = h_ab + j * ld;
      for (int t = 0; t < ld; ++t) col[t] = ie_complex{0.0, 0.0};
      for (int t = 0; t < kv; ++t) col[t] = ie_complex{U[j * kv + t].x, U[j * kv + t].y};
      col[kv] = ie_complex{D[j].x, D[j].y};
      for (int t = 0; t < k_l; ++t) col[kv + 1 + t] = ie_complex{L[j * klp + t].x, L[j * klp + t].y};
    }
  }
  if (h_ipiv) {
    CK(cudaMemcpy(h_ipiv, h->piv + (int64_t)pole * h->n_pad, sizeof(int) * (size_t)h->n,
                  cudaMemcpyDeviceToHost));
    for (int64_t i = 0; i < h->n; ++i) h_ipiv[i] += 1;   // LAPACK 1-based
  }
  return IE_OK;
}

static void fill_solve_stats(ie_handle h, ie_stats* out) {
  out->g_columns = h->g_columns;
  out->solve_launches = h->solve_launches;
  out->t_solve_ms = h->t_solve_ms;
  out->solve_flops = h->solve_flops;
  out->solve_bytes = h->solve_bytes;
  out->kernel_launches = ie_launch_count();
  out->solve32_launches = h->solve32_launches;
  out->t_solve32_ms = h->t_solve32_ms;
  out->solve32_flops = h->solve32_flops;
  out->adj_launches = h->adj_launches;
  out->t_adj_ms = h->t_adj_ms;
  out->adj_flops = h->adj_flops;
  out->refine_solves = h->refine_solves;
  out->refine_last_corr = h->refine_last_corr;
  out->solve_kernel = band_solve_last_kernel(0);
  out->solve32_kernel = band_solve_last_kernel(1);
}

extern "C" ie_status ie_get_stats(ie_handle h, ie_stats* out) {
  if (!h || !out) return IE_ERR_ARG;
  flush_solve_timing(h);
  *out = h->stats;
  fill_solve_stats(h, out);
  return IE_OK;
}

// ------------------------------ internal accessor (ie_static.cu) -----------------------------
// Read-only view of a handle's factors for entry points defined in other translation units.
bool ie_internal_factors(ie_handle h, IeFactorsView* v) {
  if (!h || !v) return false;
  v->dev = h->dev;
  v->P = h->P;
  v->n = h->n;
  v->n_pad = h->n_pad;
  v->kl = h->kl;
  v->ldab = h->ldab;
  v->q = h->q;
  v->AB = h->AB;
  v->L64 = h->L64;
  v->U64 = h->U64;
  v->piv = h->piv;
  v->dinv = h->dinv;
  v->Tb = h->Tb;
  v->Hb = h->Hb;
  v->Ub = h->Uinvb;
  v->weights = h->d_weights;
  v->status = h->status;
  return true;
}

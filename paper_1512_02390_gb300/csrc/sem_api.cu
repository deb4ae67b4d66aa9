// C ABI of the GB300 Schwarz/multigrid spectral-element solver (include/sem_schwarz.h).
//
// A handle holds the level hierarchy p_l = 2^l, l = 0..L (Sec. 3.2), the
// device tables built by the FP64 host set-up, the work vectors of every
// level, and the FP64 vectors of the MGCG iteration (Alg. 4).  Every step of
// the solve runs in the CUDA kernels of this library; the host only enqueues
// launches and, once per MGCG iteration, reads the convergence flag.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <cstring>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "kernels.h"
#include "sem_schwarz.h"
#include "setup.h"
#include "tune_cache.h"

using namespace sem;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CK(call)                                                                                     \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess)                                                                           \
      return fail(SEM_CUDA_ERROR, std::string(#call) + ": " + cudaGetErrorString(e_));              \
  } while (0)

struct Level {
  int p = 0, n_o = 0, m = 0, Nx = 0, Ny = 0;
  long nodes = 0;
  DirView<double> x64{}, y64{};
  DirView<float> x32{}, y32{};
  double* J64 = nullptr;  // interpolation from level l-1 to l
  float* J32 = nullptr;
  bool var = false;       // variable diffusivity: B(nu) operator, 1/nu_bar local solves
  VarView<double> v64{};
  VarView<float> v32{};
  double* nu_inv64 = nullptr;
  float* nu_inv32 = nullptr;
  void* u = nullptr;      // level vectors in the V-cycle type
  void* f = nullptr;
  void* r = nullptr;
  void* E = nullptr;      // element-blocked Schwarz corrections
  TuneVal tune{};         // launch shapes (autotuner): fused scatter, sweep kernel and grid
  TcWork tc{};            // stacks of the tcgen05 sweep (ngroups == 0: not available)
  FxDir fxx{}, fxy{};     // fixed-point even-odd tables (finest level; FP64 operator in integers)
};

}  // namespace

namespace sem {
// error message for sem_last_error from other translation units
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace sem

struct sem_handle {
  sem_config cfg{};
  int device = 0;
  int L = 0;
  bool mixed = false;
  bool mult = false;  // multiplicative Schwarz smoother (Alg. 1) instead of Alg. 2
  int sweep_mode = 0;
  Mesh1D mx, my;
  std::vector<Level> lev;
  CoarseView coarse{};
  std::vector<int> ns1, ns2;
  long n = 0, n_unknowns = 0;
  int nb = 1;        // independent problems stacked along y (batched solves)
  int rows_top = 0;  // node rows of one problem on the finest level
  double *u = nullptr, *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *r_old = nullptr;
  double* fi = nullptr;  // right side of the running MGCG solve (internal copy)
  double* Binv = nullptr;  // dense FP64 inverse of B_0(nu) (variable diffusivity)
  int* tc_err = nullptr;   // device flag: a tcgen05 sweep or a grid barrier gave up waiting
  // levels p_l <= 8 and the coarse solve in one persistent kernel (mixed modes)
  bool low_ok = false, low_on = false;
  LowCycle lowc{};
  // the up-leg of the V-cycle in one launch (no post-smoothing, p >= 4)
  bool chain_ok = false, chain_on = true;
  // the FP64 operator evaluated exactly in integers (Poisson operator, p >= 4)
  bool fx_ok = false, fx_on = true;
  // the whole MGCG solve as one CUDA graph: prologue + WHILE node over one iteration
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t cap = nullptr, cap2 = nullptr;
  long long graph_pro[SEM_K_NCLASS] = {}, graph_body[SEM_K_NCLASS] = {};
  int solves = 0;
  double* part = nullptr;
  PcgState st{};
  int* flags_host = nullptr;  // pinned: [0] problems still iterating
  std::vector<double> xc, yc;
  std::vector<void*> allocs;
  // tracing: launches per kernel class, optional CUDA-event timing
  long long launches[SEM_K_NCLASS] = {};
  bool prof = false;
  std::vector<cudaEvent_t> ev;  // pairs (start, end)
  std::vector<int> ev_cls;
  std::vector<int> ev_lvl;  // V-cycle level of each traced launch (-1: outside the V-cycle)
  std::vector<int> ev_nk;   // kernels in each traced launch
  int cur_level = -1;       // level the V-cycle is working on (tracing)
  int ev_used = 0;
};

namespace {

template <typename T>
int dev_alloc(sem_handle* h, T** ptr, size_t count) {
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SEM_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  h->allocs.push_back(d);
  *ptr = static_cast<T*>(d);
  return SEM_OK;
}

template <typename T, typename S>
int upload(sem_handle* h, T** ptr, const std::vector<S>& v) {
  std::vector<T> tmp(v.begin(), v.end());
  int rc = dev_alloc(h, ptr, tmp.size());
  if (rc) return rc;
  CK(cudaMemcpy(*ptr, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SEM_OK;
}

template <typename T>
int upload_dir(sem_handle* h, const Dir1D& d, DirView<T>& v) {
  v.p = d.p;
  v.n = d.n;
  v.N = d.N;
  v.periodic = d.periodic ? 1 : 0;
  v.n_o = d.n_o;
  v.m = d.m;
  std::vector<double> S, lam, w;
  for (const auto& t : d.tables) {
    S.insert(S.end(), t.S.begin(), t.S.end());
    lam.insert(lam.end(), t.lam.begin(), t.lam.end());
    w.insert(w.end(), t.w.begin(), t.w.end());
  }
  int rc;
  T *Le, *Mg, *Sd, *ld, *wd;
  int* tab;
  if ((rc = upload(h, &Le, d.Le))) return rc;
  if ((rc = upload(h, &Mg, d.Mglob))) return rc;
  if ((rc = upload(h, &tab, d.tab))) return rc;
  if ((rc = upload(h, &Sd, S))) return rc;
  if ((rc = upload(h, &ld, lam))) return rc;
  if ((rc = upload(h, &wd, w))) return rc;
  v.Le = Le;
  v.Mg = Mg;
  v.tab = tab;
  v.S = Sd;
  v.lam = ld;
  v.w = wd;
  return SEM_OK;
}

int overlap_for(const sem_config& c, int pl) {
  int n;
  switch (c.overlap_rule) {
    case SEM_OVERLAP_FIXED: n = c.overlap; break;
    case SEM_OVERLAP_FLOOR8: n = pl / 8; break;
    case SEM_OVERLAP_CEIL8: n = (pl + 7) / 8; break;
    case SEM_OVERLAP_CEIL2: n = (pl + 1) / 2; break;
    default: n = -1;
  }
  if (n < 0) return -1;
  return std::min(n, pl - 1);
}

bool valid_weight(int w) {
  return w == 1 || w == 3 || w == 5 || w == 7 || w == SEM_W_TOPHAT || w == SEM_W_ARITH || w == SEM_W_IDENTITY ||
         w == SEM_W_LEARNED;
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

constexpr int kMaxEventPairs = 1 << 15;

void prof_begin(sem_handle* h, int cls, cudaStream_t s, int kernels = 1) {
  h->launches[cls] += kernels;
  if (!h->prof || h->ev_used >= kMaxEventPairs) return;
  if ((int)h->ev.size() < 2 * (h->ev_used + 1)) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) {
      cudaGetLastError();
      h->prof = false;
      return;
    }
    h->ev.push_back(a);
    h->ev.push_back(b);
    h->ev_cls.push_back(cls);
    h->ev_lvl.push_back(-1);
    h->ev_nk.push_back(0);
  }
  h->ev_cls[h->ev_used] = cls;
  h->ev_lvl[h->ev_used] = h->cur_level;
  h->ev_nk[h->ev_used] = kernels;
  cudaEventRecord(h->ev[2 * h->ev_used], s);
}

void prof_end(sem_handle* h, cudaStream_t s) {
  if (!h->prof || h->ev_used >= kMaxEventPairs) return;
  cudaEventRecord(h->ev[2 * h->ev_used + 1], s);
  h->ev_used++;
}

// launch with tracing: count, and time with events when profiling is on
#define KL(h, cls, s, call)        \
  do {                             \
    prof_begin((h), (cls), (s));   \
    CK(call);                      \
    prof_end((h), (s));            \
  } while (0)
// the same for a launcher call that issues nk kernels
#define KLN(h, cls, nk, s, call)        \
  do {                                  \
    prof_begin((h), (cls), (s), (nk));  \
    CK(call);                           \
    prof_end((h), (s));                 \
  } while (0)

// ---- one level's smoothing (Alg. 2) --------------------------------------

template <typename T>
const DirView<T>& DX(const Level& l) {
  if constexpr (std::is_same<T, double>::value) return l.x64; else return l.x32;
}
template <typename T>
const DirView<T>& DY(const Level& l) {
  if constexpr (std::is_same<T, double>::value) return l.y64; else return l.y32;
}
template <typename T>
const T* JL(const Level& l) {
  if constexpr (std::is_same<T, double>::value) return l.J64; else return l.J32;
}
// views, vectors and tables of levels 0 .. L-1 for the fused up-leg
template <typename T>
ProlongChain<T> chain_view(const sem_handle* h) {
  ProlongChain<T> c{};
  for (int l = 0; l < h->L && l < kChainLevels; ++l) {
    c.x[l] = DX<T>(h->lev[l]);
    c.y[l] = DY<T>(h->lev[l]);
    c.u[l] = static_cast<const T*>(h->lev[l].u);
    c.J[l] = l > 0 ? JL<T>(h->lev[l]) : nullptr;
  }
  return c;
}
template <typename T>
const VarView<T>& VV(const Level& l) {
  if constexpr (std::is_same<T, double>::value) return l.v64; else return l.v32;
}
template <typename T>
const T* NUI(const Level& l) {
  if constexpr (std::is_same<T, double>::value) return l.nu_inv64; else return l.nu_inv32;
}

// out = A_l u (f null) or f - A_l u on level l; B_l(nu) when nu varies.
// With E, u is assembled from the Schwarz corrections (fused scatter) and
// written to uout (Poisson operator only).
// eo: -2 = the level's tuned form, else the form to use (see launch_apply).
template <typename T, typename TF = T>
int level_apply(sem_handle* h, const Level& l, int cls, const T* u, const TF* f, T* out, int dot, double* part,
                int* np, cudaStream_t s, const T* E = nullptr, T* uout = nullptr, PcgFuse pf = PcgFuse(),
                int eo = -2) {
  if (l.var) {
    if constexpr (std::is_same<T, TF>::value) {
      if (E) return fail(SEM_BAD_ARG, "fused scatter needs the Poisson operator");
      KLN(h, cls, 2, s, launch_apply_var<T>(DX<T>(l), DY<T>(l), VV<T>(l), u, f, out, dot, part, np, s));
      return SEM_OK;
    } else {
      return fail(SEM_BAD_ARG, "variable operator needs a right side of its own type");
    }
  }
  KL(h, cls, s, (launch_apply<T, TF>(DX<T>(l), DY<T>(l), u, f, out, dot, part, np, s, E, uout, pf,
                                     eo == -2 ? l.tune.eo : eo)));
  return SEM_OK;
}

// E_s = W_s A_ss^{-1} R_s r for every subdomain of level l: tcgen05 stacks or
// one subdomain per warp / CTA, as the level is tuned
template <typename T, typename TIn>
int level_sweep(sem_handle* h, const Level& l, const TIn* r, T* E, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    if (l.tune.tc && l.tc.ngroups > 0 && h->sweep_mode != 0) {
      KL(h, SEM_K_SWEEP, s,
         (launch_sweep_tc<TIn>(DX<float>(l), DY<float>(l), r, E, h->sweep_mode, NUI<float>(l), l.tc, s)));
      return SEM_OK;
    }
  }
  KL(h, SEM_K_SWEEP, s, (launch_sweep<T, TIn>(DX<T>(l), DY<T>(l), r, E, h->sweep_mode, NUI<T>(l), s, l.tune.spw)));
  return SEM_OK;
}

// u = (accum ? u : 0) + sum_s R_s^T W A_ss^{-1} R_s r  (one additive sweep on r)
template <typename T, typename TIn, typename TU>
int sweep(sem_handle* h, const Level& l, const TIn* r, TU* u, bool accum, cudaStream_t s) {
  T* E = static_cast<T*>(l.E);
  int rc = level_sweep<T, TIn>(h, l, r, E, s);
  if (rc) return rc;
  KL(h, SEM_K_SCATTER, s, (launch_scatter<T, TU>(DX<T>(l), DY<T>(l), E, u, accum, s)));
  return SEM_OK;
}

// n sweeps of the multiplicative Schwarz method (Alg. 1) on level l, u in
// place, local solves in T; the class order is reversed on even sweeps
template <typename T, typename TU, typename TF>
int mult_sweeps(sem_handle* h, const Level& l, const TF* f, TU* u, int n, cudaStream_t s) {
  const DirView<T>& dx = DX<T>(l);
  const DirView<T>& dy = DY<T>(l);
  const int nk = std::min(mult_colours(dx.n, dx.periodic != 0), dx.n) *
                 std::min(mult_colours(dy.n, dy.periodic != 0), dy.n);
  for (int i = 1; i <= n; ++i)
    KLN(h, SEM_K_SWEEP, nk, s, (launch_mult_sweep<T, TU, TF>(dx, dy, u, f, i % 2 == 0, s, nullptr)));
  return SEM_OK;
}

// n Schwarz steps from u = 0: the first residual is f itself
template <typename T>
int smooth_from_zero(sem_handle* h, const Level& l, const T* f, T* u, int n, cudaStream_t s) {
  if (n <= 0 || h->mult) {
    CK(cudaMemsetAsync(u, 0, l.nodes * sizeof(T), s));
    if (h->mult) return mult_sweeps<T, T, T>(h, l, f, u, n, s);
    return SEM_OK;
  }
  int rc = sweep<T, T, T>(h, l, f, u, false, s);
  if (rc) return rc;
  T* r = static_cast<T*>(l.r);
  for (int k = 1; k < n; ++k) {
    if ((rc = level_apply<T>(h, l, SEM_K_APPLY_MG, u, f, r, 0, nullptr, nullptr, s))) return rc;
    if ((rc = sweep<T, T, T>(h, l, r, u, true, s))) return rc;
  }
  return SEM_OK;
}

template <typename T, typename TF = T>
int smooth(sem_handle* h, const Level& l, const TF* f, T* u, int n, cudaStream_t s) {
  if (h->mult) return mult_sweeps<T, T, TF>(h, l, f, u, n, s);
  T* r = static_cast<T*>(l.r);
  for (int k = 0; k < n; ++k) {
    int rc = level_apply<T, TF>(h, l, SEM_K_APPLY_MG, u, f, r, 0, nullptr, nullptr, s);
    if (rc) return rc;
    rc = sweep<T, T, T>(h, l, r, u, true, s);
    if (rc) return rc;
  }
  return SEM_OK;
}

// One level of the down-sweep from u_l = 0 with one smoothing step: the
// sweep writes the corrections E; the residual kernel assembles u_l from E
// (scatter fused) and writes r_l = f_l - A_l u_l.
template <typename T, typename TF>
int level_down_fused(sem_handle* h, const Level& l, const TF* f, T* u, cudaStream_t s) {
  T* E = static_cast<T*>(l.E);
  T* r = static_cast<T*>(l.r);
  int rc = level_sweep<T, TF>(h, l, f, E, s);
  if (rc) return rc;
  return level_apply<T, TF>(h, l, SEM_K_APPLY_MG, nullptr, f, r, 0, nullptr, nullptr, s, E, u);
}

// z = MultigridCycle(0, rtop), Alg. 3, with the level vectors in type T.  In
// the mixed mode the finest level's right side is rtop rounded to FP32 in
// lv[L].f: written here, or already by the residual update of the outer
// iteration (r32_ready).  Every finest-level kernel rounds its right side to
// FP32 on reading, so the copy changes no result; it halves their reads and
// takes the conversions out of them.
// dot != null: the launch that writes the final z also forms z.q, z.r and
// beta (PcgDot) where it can (the finest prolongation, when no
// post-smoothing follows); *dotted tells whether it did.
template <typename T>
int vcycle_z(sem_handle* h, const double* rtop, double* zout, cudaStream_t s, bool r32_ready = false,
             const PcgDot* dot = nullptr, bool* dotted = nullptr) {
  const int L = h->L;
  auto& lv = h->lev;
  constexpr bool dbl = std::is_same<T, double>::value;
  const bool convert_top = !dbl;
  if (convert_top && !r32_ready)
    KL(h, SEM_K_VECTOR, s, (launch_convert<double, float>(lv[L].nodes, rtop, static_cast<float*>(lv[L].f), s)));
  T* uL = dbl ? reinterpret_cast<T*>(zout) : static_cast<T*>(lv[L].u);
  int rc;
  // levels 1 .. low run in the persistent kernel (0: none)
  const int low = (!dbl && h->low_ok && h->low_on) ? h->lowc.top : 0;
  struct LevelTag {  // tracing: launches inside the cycle carry their level
    sem_handle* h;
    ~LevelTag() { h->cur_level = -1; }
  } tag{h};
  for (int l = L; l >= 1 && l > low; --l) {
    h->cur_level = l;
    T* ul = (l == L) ? uL : static_cast<T*>(lv[l].u);
    T* rl = static_cast<T*>(lv[l].r);
    const bool fuse = lv[l].tune.fuse && h->ns1[l] == 1 && !lv[l].var && !h->mult;
    if (l == L && !convert_top) {  // right side rtop (FP64)
      if (fuse) {
        if ((rc = level_down_fused<T, double>(h, lv[l], rtop, ul, s))) return rc;
      } else {
        if constexpr (dbl) {
          if ((rc = smooth_from_zero<T>(h, lv[l], rtop, ul, h->ns1[l], s))) return rc;
        } else {
          // several pre-smoothing steps from an FP64 right side: first sweep on
          // rtop itself, then residual sweeps
          if (h->ns1[l] <= 0) {
            CK(cudaMemsetAsync(ul, 0, lv[l].nodes * sizeof(T), s));
          } else {
            if ((rc = sweep<T, double, T>(h, lv[l], rtop, ul, false, s))) return rc;
            if ((rc = smooth<T, double>(h, lv[l], rtop, ul, h->ns1[l] - 1, s))) return rc;
          }
        }
        if ((rc = level_apply<T, double>(h, lv[l], SEM_K_APPLY_MG, ul, rtop, rl, 0, nullptr, nullptr, s))) return rc;
      }
    } else {
      const T* fl = static_cast<const T*>(lv[l].f);
      if (fuse) {
        if ((rc = level_down_fused<T, T>(h, lv[l], fl, ul, s))) return rc;
      } else {
        if ((rc = smooth_from_zero<T>(h, lv[l], fl, ul, h->ns1[l], s))) return rc;
        if ((rc = level_apply<T>(h, lv[l], SEM_K_APPLY_MG, ul, fl, rl, 0, nullptr, nullptr, s))) return rc;
      }
    }
    KL(h, SEM_K_RESTRICT, s,
       launch_restrict<T>(DX<T>(lv[l]), DY<T>(lv[l]), DX<T>(lv[l - 1]), DY<T>(lv[l - 1]), JL<T>(lv[l]), rl,
                          static_cast<T*>(lv[l - 1].f), s));
  }
  h->cur_level = low ? low : 0;
  if (low) {
    KL(h, SEM_K_LOW_CYCLE, s, launch_low_cycle(h->lowc, h->sweep_mode, 1 << low, nullptr, s));
  } else if (h->Binv) {
    KL(h, SEM_K_COARSE, s,
       launch_coarse_dense<T>(h->coarse, h->Binv, static_cast<const T*>(lv[0].f), static_cast<T*>(lv[0].u), s));
  } else {
    KLN(h, SEM_K_COARSE, coarse_launches(h->coarse, !dbl), s,
        launch_coarse<T>(h->coarse, static_cast<const T*>(lv[0].f), static_cast<T*>(lv[0].u), s));
  }
  bool z_written = dbl;
  // without post-smoothing the finest level's launch carries the whole up-leg
  const bool chain = low == 0 && h->chain_ok && h->chain_on;
  for (int l = low + 1; l <= L; ++l) {
    h->cur_level = l;
    if (chain && l < L) continue;
    T* ul = (l == L) ? uL : static_cast<T*>(lv[l].u);
    const T* uc = static_cast<const T*>(lv[l - 1].u);
    if (chain) {
      const bool with_dot = dot && dot->gyp > 0;
      KL(h, SEM_K_PROLONG, s,
         (launch_prolong_chain<T>(chain_view<T>(h), DX<T>(lv[L]), DY<T>(lv[L]), JL<T>(lv[L]), ul, zout,
                                  with_dot ? dot : nullptr, s)));
      z_written = true;
      if (with_dot) *dotted = true;
      continue;
    }
    if (dot && l == L && h->ns2[l] == 0 && dot->gyp > 0) {
      // z = (dbl: ul +) I uc, with the dot products
      KL(h, SEM_K_PROLONG, s,
         (launch_prolong_dot<T>(DX<T>(lv[l]), DY<T>(lv[l]), DX<T>(lv[l - 1]), DY<T>(lv[l - 1]), JL<T>(lv[l]), uc,
                                ul, zout, *dot, s)));
      z_written = true;
      *dotted = true;
      continue;
    }
    if (l == L && !z_written && h->ns2[l] == 0) {
      KL(h, SEM_K_PROLONG, s,
         (launch_prolong<T, double>(DX<T>(lv[l]), DY<T>(lv[l]), DX<T>(lv[l - 1]), DY<T>(lv[l - 1]), JL<T>(lv[l]),
                                    uc, ul, zout, s)));
      z_written = true;
      continue;
    }
    KL(h, SEM_K_PROLONG, s,
       (launch_prolong<T, T>(DX<T>(lv[l]), DY<T>(lv[l]), DX<T>(lv[l - 1]), DY<T>(lv[l - 1]), JL<T>(lv[l]), uc, ul,
                             ul, s)));
    if (h->ns2[l] > 0) {
      if (l == L && !convert_top) {
        if ((rc = smooth<T, double>(h, lv[l], rtop, ul, h->ns2[l], s))) return rc;
      } else {
        if ((rc = smooth<T>(h, lv[l], static_cast<const T*>(lv[l].f), ul, h->ns2[l], s))) return rc;
      }
    }
  }
  if (!z_written) KL(h, SEM_K_VECTOR, s, (launch_convert<float, double>(lv[L].nodes, static_cast<const float*>(lv[L].u), zout, s)));
  return SEM_OK;
}

// r32_ready: the FP32 copy of r sits in the finest level's f (mixed mode)
int precond(sem_handle* h, const double* r, double* z, cudaStream_t s, bool r32_ready = false,
            const PcgDot* dot = nullptr, bool* dotted = nullptr) {
  if (dotted) *dotted = false;
  return h->mixed ? vcycle_z<float>(h, r, z, s, r32_ready, dot, dotted)
                  : vcycle_z<double>(h, r, z, s, false, dot, dotted);
}

const Level& top(const sem_handle* h) { return h->lev[h->L]; }

// The FP64 operator of the outer iteration: it defines the discrete problem.
// Where the fixed-point tables exist (Poisson operator, p >= 4) it runs in
// exact integer arithmetic (launch_apply_fx): the even-odd folding is exact
// there and the products are rounded once.  Otherwise, in FP64 mode, it
// applies the element matrices as stored (eo = 0): the FP64 even-odd form folds
// them into (L_ak +- L_a,p-k) / 2, whose roundings move the coefficients by up
// to half an ulp, and the exact discrete solution with them (by about 1e-11
// relative at 64 x 64 elements, p = 16); the mixed modes, whose solution bar
// is 1e-9, keep that form.
int apply64(sem_handle* h, const double* u, const double* f, double* out, int dot, int* np, cudaStream_t s,
            double* part = nullptr, PcgFuse pf = PcgFuse()) {
  const Level& t = top(h);
  if (h->fx_ok && h->fx_on) {
    KL(h, SEM_K_APPLY_FP64, s,
       launch_apply_fx(DX<double>(t), DY<double>(t), t.fxx, t.fxy, u, f, out, dot, part ? part : h->part, np, s,
                       pf));
    return SEM_OK;
  }
  return level_apply<double>(h, t, SEM_K_APPLY_FP64, u, f, out, dot, part ? part : h->part, np, s, nullptr,
                             nullptr, pf, h->mixed ? -2 : 0);
}

// Tile rows per problem of the finest prolongation when it can form the
// z.q, z.r partials (PcgDot), else 0: one problem (any height), or stacked
// problems whose tiles do not straddle two; 2 x tiles <= kMaxPartials.
int dot_tile_rows(const sem_handle* h) {
  const Level& t = top(h);
  const int te = tile_elems(t.p), ny = t.y64.n, nyp = ny / h->nb;
  const long nct = prolong_ctas(t.p, t.x64.n, ny);
  if (nct <= 0 || 2 * nct > kMaxPartials) return 0;
  if (h->nb == 1) return (ny + te - 1) / te;
  return (nyp * h->nb == ny && nyp % te == 0) ? nyp / te : 0;
}

// The direction update p = z + beta p of Alg. 4 fused into the FP64 operator
// and the u, r update (Poisson operator): beta from the z.q, z.r reduction.
bool fused_direction(const sem_handle* h) { return !top(h).var; }

// ---- MGCG, Alg. 4, on the internal vectors h->u, h->fi ---------------------
// Iteration i is split as: [V-cycle z = M r_{i-1}; beta; p] (body start) and
// [q = A p; alpha; u, r; ||r|| test] (body end), so the convergence test ends
// the body and the loop needs no nested condition.  Iteration 1's second half
// belongs to the prologue.

// q = A p, p.q;  u, r update and the fused convergence check.  fused: the
// operand is z + beta p (stored as the new p by the update kernel)
int pcg_tail(sem_handle* h, cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond, bool fused) {
  int np = 0, rc;
  PcgFuse pf;
  if (fused) {
    pf.z = h->z;
    pf.beta = h->st.beta;
    pf.flags = h->st.flags;
    pf.iter = h->st.iter;
    pf.stride = h->st.stride;
    pf.nb = h->nb;
  }
  if ((rc = apply64(h, h->p, nullptr, h->q, 1, &np, s, nullptr, pf))) return rc;
  KL(h, SEM_K_VECTOR, s,
     launch_pcg_update_ur_check(h->n, h->u, h->r, h->p, h->q, h->part, np / h->nb, h->st, h->part + kMaxPartials,
                                h->cfg.i_max, cond, use_cond, s, fused ? h->z : nullptr,
                                h->mixed ? static_cast<float*>(top(h).f) : nullptr));
  return SEM_OK;
}

int pcg_prologue(sem_handle* h, cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond) {
  const long n = h->n;
  int np = 0, rc;
  // r = f - A u and ||r_0||^2 partials
  if ((rc = apply64(h, h->u, h->fi, h->r, 2, &np, s, h->part + 2 * kMaxPartials))) return rc;
  // p = MultigridCycle(0, r); delta = p.r; r_old = 0
  if ((rc = precond(h, h->r, h->z, s))) return rc;
  KL(h, SEM_K_VECTOR, s, launch_dot2(n, h->z, h->r, h->r, h->part, h->st, s));
  KLN(h, SEM_K_VECTOR, 2, s,
      launch_pcg_start(n, h->z, h->r, h->p, h->r_old, h->part, h->part + 2 * kMaxPartials, np / h->nb, h->st,
                       h->cfg.tol, s));
  return pcg_tail(h, s, cond, use_cond, false);
}

int pcg_body(sem_handle* h, cudaStream_t s, cudaGraphConditionalHandle cond, int use_cond) {
  const long n = h->n;
  int rc;
  // the previous body's (or the prologue's) update kernel wrote r's FP32 copy
  if (fused_direction(h)) {
    // the V-cycle's last launch forms z.q, z.r and beta (per stacked problem)
    const PcgDot dot = {h->q, h->r, h->part, h->st, dot_tile_rows(h)};
    bool dotted = false;
    if ((rc = precond(h, h->r, h->z, s, true, dot.gyp > 0 ? &dot : nullptr, &dotted))) return rc;
    if (!dotted) KL(h, SEM_K_VECTOR, s, launch_dot2_beta(n, h->z, h->r, h->q, h->part, h->st, s));
    return pcg_tail(h, s, cond, use_cond, true);
  }
  if ((rc = precond(h, h->r, h->z, s, true))) return rc;
  KL(h, SEM_K_VECTOR, s, launch_dot2(n, h->z, h->r, h->r_old, h->part, h->st, s));
  KL(h, SEM_K_VECTOR, s, launch_pcg_update_p(n, h->z, h->p, h->r, h->r_old, h->part, h->st, s));
  return pcg_tail(h, s, cond, use_cond, false);
}

// Add prologue + WHILE(body) of h's MGCG to the capture running on `cap`
// (body captured through `cap2`); the body's last kernel sets the condition.
// Launch counts of the captured prologue / body are kept for the tracing
// counters of graph replays.
int capture_solve(sem_handle* h, cudaStream_t cap, cudaStream_t cap2) {
  long long before[SEM_K_NCLASS];
  for (int c = 0; c < SEM_K_NCLASS; ++c) before[c] = h->launches[c];
  cudaStreamCaptureStatus cs;
  cudaGraph_t capg = nullptr;
  CK(cudaStreamGetCaptureInfo(cap, &cs, nullptr, &capg, nullptr, nullptr, nullptr));
  cudaGraphConditionalHandle cond;
  CK(cudaGraphConditionalHandleCreate(&cond, capg, 0, 0));
  int rc = pcg_prologue(h, cap, cond, 1);
  if (rc) return rc;
  for (int c = 0; c < SEM_K_NCLASS; ++c) h->graph_pro[c] = h->launches[c] - before[c];
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  CK(cudaStreamGetCaptureInfo(cap, &cs, nullptr, &capg, &deps, nullptr, &nd));
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = cond;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t cnode;
  CK(cudaGraphAddNode(&cnode, capg, deps, nullptr, nd, &cp));
  CK(cudaStreamUpdateCaptureDependencies(cap, &cnode, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t body = cp.conditional.phGraph_out[0];
  for (int c = 0; c < SEM_K_NCLASS; ++c) before[c] = h->launches[c];
  CK(cudaStreamBeginCaptureToGraph(cap2, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  rc = pcg_body(h, cap2, cond, 1);
  cudaGraph_t body_out = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cap2, &body_out);
  if (rc) return rc;
  if (e2 != cudaSuccess) return fail(SEM_CUDA_ERROR, "body capture failed");
  for (int c = 0; c < SEM_K_NCLASS; ++c) {
    h->graph_body[c] = h->launches[c] - before[c];
    h->launches[c] -= h->graph_pro[c] + h->graph_body[c];
  }
  return SEM_OK;
}

int end_capture_discard(cudaStream_t cap) {
  cudaGraph_t junk = nullptr;
  cudaStreamEndCapture(cap, &junk);
  if (junk) cudaGraphDestroy(junk);
  cudaGetLastError();
  return 0;
}

int build_graph(sem_handle* h) {
  CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  CK(cudaStreamCreateWithFlags(&h->cap2, cudaStreamNonBlocking));
  CK(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeRelaxed));
  int rc = capture_solve(h, h->cap, h->cap2);
  if (rc) {
    end_capture_discard(h->cap);
    return rc;
  }
  CK(cudaStreamEndCapture(h->cap, &h->graph));
  CK(cudaGraphInstantiate(&h->graph_exec, h->graph, 0));
  return SEM_OK;
}

// read and clear the tcgen05 give-up flag (sync)
int take_tc_err(sem_handle* h, cudaStream_t s, bool& hit) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  hit = e != 0;
  if (hit) {
    CK(cudaMemsetAsync(h->tc_err, 0, sizeof(int), s));
    if (h->lowc.bar) CK(cudaMemsetAsync(h->lowc.bar, 0, 2 * sizeof(unsigned), s));
  }
  return SEM_OK;
}

// host copy of the number of problems still iterating
int sync_flags(sem_handle* h, cudaStream_t s) {
  CK(cudaMemcpyAsync(h->flags_host, h->st.active, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return SEM_OK;
}

int check_handle(const sem_handle* h) {
  if (!h) return fail(SEM_BAD_ARG, "null handle");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device) {
    cudaGetLastError();
    return fail(SEM_BAD_ARG, "the current CUDA device is not the handle's device");
  }
  return SEM_OK;
}

// drop the captured solve graph (launch shapes changed): the next solve
// captures a new one
void drop_graph(sem_handle* h) {
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->cap2) cudaStreamDestroy(h->cap2);
  h->graph_exec = nullptr;
  h->graph = nullptr;
  h->cap = h->cap2 = nullptr;
}

// one down-sweep step of level l from u_l = 0 (one pre-smoothing sweep, then
// the level residual) with the level's current launch shapes
template <typename T, typename TF>
int down_step(sem_handle* h, Level& l, const TF* f, T* u, cudaStream_t s) {
  if (l.tune.fuse) return level_down_fused<T, TF>(h, l, f, u, s);
  int rc = sweep<T, TF, T>(h, l, f, u, false, s);
  if (rc) return rc;
  return level_apply<T, TF>(h, l, SEM_K_APPLY_MG, u, f, static_cast<T*>(l.r), 0, nullptr, nullptr, s);
}

// Time every launch-shape candidate of level l on the level's own vectors
// (best of three batches of ten steps each) and keep the fastest.
template <typename T, typename TF>
int tune_level(sem_handle* h, Level& l, const TF* f, bool allow_fuse, cudaStream_t s, cudaEvent_t e0,
               cudaEvent_t e1) {
  T* u = static_cast<T*>(l.u);
  const bool mma = std::is_same<T, float>::value && h->sweep_mode != 0;
  // sweep kernels: (tc, spw) = tcgen05 stacks, or mma.sync with 1, 2, 4 subdomains per warp
  std::vector<std::pair<int, int>> kern = {{0, 1}};
  if (mma) {
    kern.push_back({0, 2});
    kern.push_back({0, 4});
    if (l.tc.ngroups > 0) kern.push_back({1, 1});
  }
  TuneVal best;
  best.us = -1.0;
  constexpr int kReps = 10;
  for (int fuse = 0; fuse <= (allow_fuse ? 1 : 0); ++fuse)
    for (const auto& kc : kern) {
      l.tune.fuse = fuse;
      l.tune.tc = kc.first;
      l.tune.spw = kc.second;
      int rc;
      for (int w = 0; w < 2; ++w)
        if ((rc = down_step<T, TF>(h, l, f, u, s))) return rc;
      double us = -1.0;
      for (int batch = 0; batch < 3; ++batch) {
        CK(cudaEventRecord(e0, s));
        for (int r = 0; r < kReps; ++r)
          if ((rc = down_step<T, TF>(h, l, f, u, s))) return rc;
        CK(cudaEventRecord(e1, s));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        const double t = 1000.0 * ms / kReps;
        if (us < 0 || t < us) us = t;
      }
      if (best.us < 0 || us < best.us) best = l.tune, best.us = us;
    }
  // then the residual's form: the even-odd operator in FP32 (P >= 4)
  if (std::is_same<T, float>::value && l.p >= 4) {
    l.tune = best;
    l.tune.eo = 1;
    int rc;
    for (int w = 0; w < 2; ++w)
      if ((rc = down_step<T, TF>(h, l, f, u, s))) return rc;
    double us = -1.0;
    for (int batch = 0; batch < 3; ++batch) {
      CK(cudaEventRecord(e0, s));
      for (int r = 0; r < kReps; ++r)
        if ((rc = down_step<T, TF>(h, l, f, u, s))) return rc;
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      const double t = 1000.0 * ms / kReps;
      if (us < 0 || t < us) us = t;
    }
    if (us < best.us) best = l.tune, best.us = us;
  }
  l.tune = best;
  return SEM_OK;
}

// tune (or read from the cache) every level l = 1..L of h on stream s
int autotune(sem_handle* h, const std::string& path, cudaStream_t s) {
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, h->device));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return fail(SEM_CUDA_ERROR, "cudaEventCreate failed");
  }
  long long saved[SEM_K_NCLASS];
  std::memcpy(saved, h->launches, sizeof(saved));
  const bool prof = h->prof;
  h->prof = false;
  int rc = SEM_OK;
  for (int l = 1; l <= h->L && rc == SEM_OK; ++l) {
    Level& lv = h->lev[l];
    const std::string key = tune_key(prop.name, lv.p, lv.n_o, h->cfg.precision, lv.var ? 1 : 0, lv.x64.n, lv.y64.n);
    TuneVal v;
    if (!path.empty() && tune_cache_find(path, key, v) && !(v.tc && lv.tc.ngroups == 0)) {
      lv.tune = v;
      continue;
    }
    const bool allow_fuse = h->ns1[l] == 1 && !lv.var && !h->mult;
    if (!allow_fuse && !(h->mixed && h->sweep_mode != 0)) {
      lv.tune = TuneVal{};  // a single candidate: nothing to time
    } else if (!h->mixed) {
      rc = tune_level<double, double>(h, lv, static_cast<const double*>(lv.f), allow_fuse, s, e0, e1);
    } else if (l == h->L && !lv.var) {  // the mixed V-cycle reads the FP64 residual here
      if (cudaMemsetAsync(h->r, 0, h->n * sizeof(double), s) != cudaSuccess) rc = fail(SEM_CUDA_ERROR, "memset");
      if (!rc) rc = tune_level<float, double>(h, lv, h->r, allow_fuse, s, e0, e1);
    } else {
      rc = tune_level<float, float>(h, lv, static_cast<const float*>(lv.f), allow_fuse, s, e0, e1);
    }
    if (!rc && !path.empty()) {
      const std::string err = tune_cache_store(path, key, lv.tune);
      if (!err.empty()) rc = fail(SEM_BAD_ARG, err);
    }
  }
  // the persistent low-level cycle against the per-level launches: whole
  // V-cycles on the FP64 residual buffer, best of 3 x 10
  if (!rc && h->low_ok) {
    const std::string key = std::string(prop.name) + "|low-cycle|p=" + std::to_string(h->cfg.p) + "|n_o=" +
                            std::to_string(h->lev[h->L].n_o) + "|prec=" + std::to_string(h->cfg.precision) +
                            "|elems=" + std::to_string(h->lev[h->L].x64.n) + "x" + std::to_string(h->lev[h->L].y64.n);
    TuneVal v;
    if (!path.empty() && tune_cache_find(path, key, v)) {
      h->low_on = v.fuse != 0;
    } else {
      double best_us[2] = {-1.0, -1.0};
      for (int on = 0; on <= 1 && !rc; ++on) {
        h->low_on = on != 0;
        for (int w = 0; w < 2 && !rc; ++w) rc = precond(h, h->r, h->z, s);
        for (int batch = 0; batch < 3 && !rc; ++batch) {
          if (cudaEventRecord(e0, s) != cudaSuccess) rc = fail(SEM_CUDA_ERROR, "event");
          for (int r = 0; r < 10 && !rc; ++r) rc = precond(h, h->r, h->z, s);
          if (!rc && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
            rc = fail(SEM_CUDA_ERROR, "event");
          float ms = 0.f;
          if (!rc && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = fail(SEM_CUDA_ERROR, "event");
          const double t = 100.0 * ms;  // microseconds per V-cycle
          if (!rc && (best_us[on] < 0 || t < best_us[on])) best_us[on] = t;
        }
      }
      if (!rc) {
        h->low_on = best_us[1] < best_us[0];
        v = TuneVal{};
        v.fuse = h->low_on ? 1 : 0;
        v.us = h->low_on ? best_us[1] : best_us[0];
        if (!path.empty()) {
          const std::string err = tune_cache_store(path, key, v);
          if (!err.empty()) rc = fail(SEM_BAD_ARG, err);
        }
      }
    }
  }
  if (cudaStreamSynchronize(s) != cudaSuccess && !rc) rc = fail(SEM_CUDA_ERROR, "autotune stream failed");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  std::memcpy(h->launches, saved, sizeof(saved));
  h->prof = prof;
  drop_graph(h);
  return rc;
}

}  // namespace

extern "C" {

void sem_default_config(sem_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->nx = c->ny = 4;
  c->p = 4;
  c->periodic = 0;
  c->lx = c->ly = 1.0;
  c->overlap_rule = SEM_OVERLAP_FIXED;
  c->overlap = 1;
  c->weight = SEM_W_QUINTIC;
  c->ns1 = 1;
  c->ns2 = 0;
  c->variable_cycle = 0;
  c->precision = SEM_PREC_FP64;
  c->tol = 1e-10;
  c->i_max = 200;
}

const char* sem_status_string(int32_t s) {
  switch (s) {
    case SEM_OK: return "SEM_OK";
    case SEM_NOT_CONVERGED: return "SEM_NOT_CONVERGED";
    case SEM_BREAKDOWN: return "SEM_BREAKDOWN";
    case SEM_TIMEOUT: return "SEM_TIMEOUT";
    case SEM_BAD_ARG: return "SEM_BAD_ARG";
    case SEM_CUDA_ERROR: return "SEM_CUDA_ERROR";
    case SEM_OOM: return "SEM_OOM";
    default: return "unknown";
  }
}

const char* sem_last_error(void) { return g_err.c_str(); }

void sem_destroy(sem_handle* h) {
  if (!h) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  if (h->graph_exec) cudaGraphExecDestroy(h->graph_exec);
  if (h->graph) cudaGraphDestroy(h->graph);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->cap2) cudaStreamDestroy(h->cap2);
  for (void* p : h->allocs) cudaFree(p);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  if (h->flags_host) cudaFreeHost(h->flags_host);
  if (prev >= 0) cudaSetDevice(prev);
  cudaGetLastError();
  delete h;
}

static int validate(const sem_config& c, int& L) {
  L = 0;
  while ((1 << L) < c.p) ++L;
  if (c.p < 2 || c.p > 32 || (1 << L) != c.p) return fail(SEM_BAD_ARG, "p must be a power of two in [2, 32]");
  if (c.nx < 2 || c.ny < 2 || c.nx > 4096 || c.ny > 4096) return fail(SEM_BAD_ARG, "nx, ny must be in [2, 4096]");
  if (!valid_weight(c.weight)) return fail(SEM_BAD_ARG, "unknown weight function");
  if (c.overlap_rule < 0 || c.overlap_rule > 3 || (c.overlap_rule == SEM_OVERLAP_FIXED && c.overlap < 0))
    return fail(SEM_BAD_ARG, "invalid overlap rule");
  if (c.precision < 0 || c.precision > 3) return fail(SEM_BAD_ARG, "invalid precision");
  if (c.ns1 < 0 || c.ns2 < 0 || c.ns1 + c.ns2 < 1 || c.ns1 > 64 || c.ns2 > 64)
    return fail(SEM_BAD_ARG, "need 0 <= ns1, ns2 <= 64 and ns1 + ns2 >= 1");
  if (!(c.tol >= 0.0) || c.i_max < 1 || c.i_max > 100000) return fail(SEM_BAD_ARG, "invalid tol or i_max");
  if (c.nu_kind < 0 || c.nu_kind > 2) return fail(SEM_BAD_ARG, "unknown nu_kind");
  if (c.weight == SEM_W_LEARNED) {
    if (!c.learned_x || !c.learned_y) return fail(SEM_BAD_ARG, "learned weights need learned_x and learned_y");
    for (int lvl = 0; lvl <= L; ++lvl)
      for (int dir = 0; dir < 2; ++dir) {
        const int n = dir ? c.ny : c.nx;
        const double* a = (dir ? c.learned_y : c.learned_x) + (size_t)lvl * (n + 1) * 2;
        for (int i = 0; i <= n; ++i)
          if (!(a[2 * i] > 0.0 && a[2 * i] <= 1.0) || !(a[2 * i + 1] >= 1.0 && a[2 * i + 1] <= 7.0))
            return fail(SEM_BAD_ARG, "learned (s, kt) must satisfy 0 < s <= 1, 1 <= kt <= 7");
      }
  }
  if (c.nu_kind && c.periodic && (long)c.nx * c.ny > 1024)
    return fail(SEM_BAD_ARG, "periodic variable diffusivity: at most 32 x 32 elements (dense coarse pseudo-inverse)");
  if (c.smoother != SEM_SMOOTH_ADDITIVE && c.smoother != SEM_SMOOTH_MULT) return fail(SEM_BAD_ARG, "unknown smoother");
  if (c.smoother == SEM_SMOOTH_MULT) {
    if (c.precision != SEM_PREC_FP64 && c.precision != SEM_PREC_FP32)
      return fail(SEM_BAD_ARG, "the multiplicative smoother runs in FP64 or FP32 precision");
    if (c.nu_kind) return fail(SEM_BAD_ARG, "the multiplicative smoother needs the Poisson operator (nu_kind 0)");
    if (c.periodic && (c.nx < 3 || c.ny < 3))
      return fail(SEM_BAD_ARG, "the multiplicative smoother needs n >= 3 per direction on a periodic mesh");
  }
  if (c.nu_kind == 1 && !(c.nu_a >= 1.0)) return fail(SEM_BAD_ARG, "contrast must be >= 1");
  if (c.nu_kind == 2 && !(std::fabs(c.nu_a) < 1.0)) return fail(SEM_BAD_ARG, "amplitude must be in (-1, 1)");
  if (!c.x_edges && !(c.lx > 0)) return fail(SEM_BAD_ARG, "lx must be positive");
  if (!c.y_edges && !(c.ly > 0)) return fail(SEM_BAD_ARG, "ly must be positive");
  // the coarse solve stages one panel of up to 1024 unknowns per direction
  const int cux = c.periodic ? c.nx : c.nx - 1, cuy = c.periodic ? c.ny : c.ny - 1;
  if (cux > 1024 || cuy > 1024) return fail(SEM_BAD_ARG, "coarse grid too large (at most 1024 unknowns per direction)");
  return SEM_OK;
}

static bool make_mesh(int n, double len, const double* edges, bool periodic, Mesh1D& m) {
  m.n = n;
  m.periodic = periodic;
  m.edges.resize(n + 1);
  for (int i = 0; i <= n; ++i) m.edges[i] = edges ? edges[i] : len * i / n;
  for (int i = 0; i < n; ++i)
    if (!(m.edges[i + 1] > m.edges[i])) return false;
  return true;
}

int sem_gll_tables(int32_t p, double* xi, double* w, double* D, double* L_ref) {
  g_err.clear();
  if (p < 1 || p > 64) return fail(SEM_BAD_ARG, "need 1 <= p <= 64");
  std::vector<double> x, wq, Dm, M, L;
  gll(p, x, wq);
  gll_deriv(p, Dm);
  element_matrices(p, 2.0, M, L);  // h = 2: the reference element [-1, 1]
  const size_t n = p + 1;
  if (xi) std::memcpy(xi, x.data(), n * sizeof(double));
  if (w) std::memcpy(w, wq.data(), n * sizeof(double));
  if (D) std::memcpy(D, Dm.data(), n * n * sizeof(double));
  if (L_ref) std::memcpy(L_ref, L.data(), n * n * sizeof(double));
  return SEM_OK;
}

int sem_inspect_level(const sem_config* cfg, int32_t level, sem_level_info* info, int32_t* tab_x, double* S_x,
                      double* lam_x, double* w_x, double* coords_x) {
  g_err.clear();
  if (!cfg || !info) return fail(SEM_BAD_ARG, "null argument");
  int L, rc;
  if ((rc = validate(*cfg, L))) return rc;
  if (level < 1 || level > L) return fail(SEM_BAD_ARG, "level must be in [1, L]");
  Mesh1D mx;
  if (!make_mesh(cfg->nx, cfg->lx, cfg->x_edges, cfg->periodic != 0, mx)) return fail(SEM_BAD_ARG, "mesh edges must increase");
  const int p = 1 << level;
  const int no = overlap_for(*cfg, p);
  Dir1D d;
  const double* lx = cfg->learned_x ? cfg->learned_x + (size_t)level * (cfg->nx + 1) * 2 : nullptr;
  std::string err = build_dir(mx, p, no, cfg->weight, d, lx);
  if (!err.empty()) return fail(SEM_BAD_ARG, err);
  info->p = p;
  info->n_o = no;
  info->m = d.m;
  info->n_tables_x = (int)d.tables.size();
  info->nx_nodes = d.N;
  const int m = d.m;
  for (size_t t = 0; t < d.tables.size(); ++t) {
    if (S_x) std::memcpy(S_x + t * m * m, d.tables[t].S.data(), m * m * sizeof(double));
    if (lam_x) std::memcpy(lam_x + t * m, d.tables[t].lam.data(), m * sizeof(double));
    if (w_x) std::memcpy(w_x + t * m, d.tables[t].w.data(), m * sizeof(double));
  }
  if (tab_x)
    for (int e = 0; e < d.n; ++e) tab_x[e] = d.tab[e];
  if (coords_x) std::memcpy(coords_x, d.coords.data(), d.N * sizeof(double));
  return SEM_OK;
}

int sem_learned_features(const sem_config* cfg, float* feat_x, float* feat_y) {
  g_err.clear();
  if (!cfg || !feat_x || !feat_y) return fail(SEM_BAD_ARG, "null argument");
  sem_config c = *cfg;
  if (c.weight == SEM_W_LEARNED) c.weight = SEM_W_QUINTIC;  // features do not depend on the weights
  int L, rc;
  if ((rc = validate(c, L))) return rc;
  Mesh1D mx, my;
  if (!make_mesh(c.nx, c.lx, c.x_edges, c.periodic != 0, mx) || !make_mesh(c.ny, c.ly, c.y_edges, c.periodic != 0, my))
    return fail(SEM_BAD_ARG, "mesh edges must increase");
  for (int l = 0; l <= L; ++l) {
    const int pl = 1 << l;
    const int no = l > 0 ? overlap_for(c, pl) : 0;
    std::vector<double> xi, w;
    gll(pl, xi, w);
    const double dO = xi[no + 1] + 1.0;
    std::vector<double> nub((size_t)mx.n * my.n, 1.0);
    if (c.nu_kind) {
      VarData vd;
      build_var(mx, my, pl, c.nu_kind, c.nu_a, c.nu_b, vd);
      nub = vd.nu_bar;
    }
    for (int dir = 0; dir < 2; ++dir) {
      const Mesh1D& ma = dir ? my : mx;  // direction across the line
      const Mesh1D& mb = dir ? mx : my;  // direction along the line
      float* out = (dir ? feat_y : feat_x) + (size_t)l * (ma.n + 1) * 4;
      for (int i = 0; i <= ma.n; ++i) {
        int e0 = i - 1, e1 = i;
        if (ma.periodic) {
          e0 = (e0 + ma.n) % ma.n;
          e1 = e1 % ma.n;
        }
        double ar = 1.0, rho = 1.0;
        for (int side = 0; side < 2; ++side) {
          const int e = side ? e1 : e0;
          if (e < 0 || e >= ma.n) continue;
          for (int j = 0; j < mb.n; ++j) {
            const double r = ma.h(e) / mb.h(j);
            ar = std::max(ar, std::max(r, 1.0 / r));
          }
        }
        if (e0 >= 0 && e0 < ma.n && e1 >= 0 && e1 < ma.n)
          for (int j = 0; j < mb.n; ++j) {
            const double a = dir ? nub[(size_t)e0 * mx.n + j] : nub[(size_t)j * mx.n + e0];
            const double b = dir ? nub[(size_t)e1 * mx.n + j] : nub[(size_t)j * mx.n + e1];
            rho = std::max(rho, std::max(a / b, b / a));
          }
        out[4 * i + 0] = (float)(l / 5.0);
        out[4 * i + 1] = (float)(dO / 2.0);
        out[4 * i + 2] = (float)(std::log2(ar) / 5.0);
        out[4 * i + 3] = (float)(std::log10(rho) / 2.0);
      }
    }
  }
  return SEM_OK;
}

// A handle for nb copies of the problem cfg stacked along y (nb = 1: one
// problem).  Stacked copies share every table; walls separate them.
// Stacks of the tcgen05 sweep of one level: subdomains grouped by their pair of
// table ids, G = floor(128 / m) per stack, in row-major order within a pair.
// Left unbuilt (the level keeps the per-subdomain kernels) when the stacks
// would be less than half full, e.g. on meshes stretched in both directions.
static int build_tc_work(sem_handle* h, const Dir1D& dx, const Dir1D& dy, Level& lv) {
  if (lv.m < 2 || lv.m > 64) return SEM_OK;
  const int G = 128 / lv.m;
  std::map<std::pair<int, int>, std::vector<int>> cls;
  for (int ey = 0; ey < dy.n; ++ey)
    for (int ex = 0; ex < dx.n; ++ex) cls[{dx.tab[ex], dy.tab[ey]}].push_back(ey * dx.n + ex);
  std::vector<int> sub;
  long members = 0;
  int ng = 0;
  for (const auto& kv : cls) {
    const auto& v = kv.second;
    for (size_t i = 0; i < v.size(); i += G, ++ng)
      for (int k = 0; k < G; ++k) sub.push_back(i + k < v.size() ? v[i + k] : -1);
    members += (long)v.size();
  }
  if (2 * members < (long)ng * G) return SEM_OK;
  int* d = nullptr;
  int rc = upload(h, &d, sub);
  if (rc) return rc;
  lv.tc = TcWork{d, ng, G, h->tc_err};
  lv.tune.tc = 1;
  return SEM_OK;
}

static int create_handle(const sem_config& c, int nb, sem_handle** out) {
  int L = 0;
  {
    int rc0 = validate(c, L);
    if (rc0) return rc0;
  }
  if (nb < 1) return fail(SEM_BAD_ARG, "nb must be positive");
  if (nb > 1 && (c.periodic || c.y_edges || c.nu_kind || c.weight == SEM_W_LEARNED || c.smoother != SEM_SMOOTH_ADDITIVE))
    return fail(SEM_BAD_ARG, "stacked problems must be uniform Dirichlet Poisson problems");
  if (nb > 1 && c.ny % tile_elems(c.p) != 0)
    return fail(SEM_BAD_ARG, "stacked problems need ny divisible by the operator tile height");
  if ((long)nb * c.ny > 65536) return fail(SEM_BAD_ARG, "too many stacked problems");
  auto mesh = make_mesh;
  sem_handle* h = new sem_handle();
  h->cfg = c;
  h->cfg.x_edges = h->cfg.y_edges = nullptr;
  h->cfg.learned_x = h->cfg.learned_y = nullptr;
  h->cfg.mlp_params = nullptr;
  h->nb = nb;
  Mesh1D my1;  // one problem's y mesh (coarse factors)
  if (!mesh(c.nx, c.lx, c.x_edges, c.periodic != 0, h->mx) || !mesh(c.ny, c.ly, c.y_edges, c.periodic != 0, my1) ||
      !mesh(c.ny * nb, c.ly * nb, nb > 1 ? nullptr : c.y_edges, c.periodic != 0, h->my)) {
    delete h;
    return fail(SEM_BAD_ARG, "mesh edges must increase");
  }
  if (nb > 1) h->my.seg = c.ny;
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(SEM_CUDA_ERROR, "no usable CUDA device");
  }
  h->L = L;
  h->mixed = c.precision != SEM_PREC_FP64;
  h->mult = c.smoother == SEM_SMOOTH_MULT;
  if (h->mult) {  // the largest window must fit one CTA's shared memory
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return fail(SEM_CUDA_ERROR, "cannot query the shared-memory limit");
    }
    for (int l = 1; l <= L; ++l) {
      const int pl = 1 << l, no = overlap_for(c, pl);
      const size_t need = mult_smem_bytes(pl, pl + 1 + 2 * no, h->mixed ? sizeof(float) : sizeof(double));
      if (need > (size_t)optin) {
        delete h;
        return fail(SEM_BAD_ARG, "multiplicative smoother: level p=" + std::to_string(pl) + " needs " +
                                     std::to_string(need) + " bytes of shared memory per block; the device allows " +
                                     std::to_string(optin));
      }
    }
  }
  h->sweep_mode = c.precision == SEM_PREC_TF32 ? 1 : (c.precision == SEM_PREC_BF16 ? 2 : 0);
  h->ns1.assign(L + 1, 0);
  h->ns2.assign(L + 1, 0);
  for (int l = 1; l <= L; ++l) {
    const int f = c.variable_cycle ? (1 << (L - l)) : 1;
    h->ns1[l] = c.ns1 * f;
    h->ns2[l] = c.ns2 * f;
  }
  h->chain_ok = L >= 2 && L < kChainLevels;
  for (int l = 1; l <= L; ++l) h->chain_ok = h->chain_ok && h->ns2[l] == 0;
  int rc = SEM_OK;
  auto bail = [&](int code) {
    sem_destroy(h);
    return code;
  };
  const size_t tsz = h->mixed ? sizeof(float) : sizeof(double);
  if ((rc = dev_alloc(h, &h->tc_err, 1))) return bail(rc);
  CK(cudaMemset(h->tc_err, 0, sizeof(int)));
  h->lev.resize(L + 1);
  for (int l = 0; l <= L; ++l) {
    Level& lv = h->lev[l];
    lv.p = 1 << l;
    lv.n_o = l > 0 ? overlap_for(c, lv.p) : 0;
    lv.m = lv.p + 1 + 2 * lv.n_o;
    Dir1D dx, dy;
    const double* lx = c.learned_x ? c.learned_x + (size_t)l * (c.nx + 1) * 2 : nullptr;
    const double* ly = c.learned_y ? c.learned_y + (size_t)l * (c.ny + 1) * 2 : nullptr;
    std::string err = build_dir(h->mx, lv.p, lv.n_o, l > 0 ? c.weight : SEM_W_IDENTITY, dx, lx);
    if (err.empty()) err = build_dir(h->my, lv.p, lv.n_o, l > 0 ? c.weight : SEM_W_IDENTITY, dy, ly);
    if (!err.empty()) {
      sem_destroy(h);
      return fail(SEM_BAD_ARG, "level p=" + std::to_string(lv.p) + ": " + err);
    }
    lv.Nx = dx.N;
    lv.Ny = dy.N;
    lv.nodes = (long)dx.N * dy.N;
    if ((rc = upload_dir(h, dx, lv.x64)) || (rc = upload_dir(h, dy, lv.y64)) || (rc = upload_dir(h, dx, lv.x32)) ||
        (rc = upload_dir(h, dy, lv.y32)))
      return bail(rc);
    if (nb > 1) lv.y64.segN = lv.y32.segN = c.ny * lv.p;
    if (l > 0 && h->sweep_mode != 0 && (rc = build_tc_work(h, dx, dy, lv))) return bail(rc);
    if (l > 0) {
      std::vector<double> J;
      interp_matrix(lv.p, lv.p / 2, J);
      if ((rc = upload(h, &lv.J64, J)) || (rc = upload(h, &lv.J32, J))) return bail(rc);
    }
    if (l == L) {
      h->xc = dx.coords;
      h->yc = dy.coords;
      std::vector<int> tx, ex, sx, ty, ey, sy;
      if (lv.p >= 4 && !c.nu_kind && fx_tables(dx, tx, ex, sx) && fx_tables(dy, ty, ey, sy)) {
        int *dtx, *dex, *dsx, *dty, *dey, *dsy;
        if ((rc = upload(h, &dtx, tx)) || (rc = upload(h, &dex, ex)) || (rc = upload(h, &dsx, sx)) ||
            (rc = upload(h, &dty, ty)) || (rc = upload(h, &dey, ey)) || (rc = upload(h, &dsy, sy)))
          return bail(rc);
        lv.fxx = FxDir{dtx, dex, dsx};
        lv.fxy = FxDir{dty, dey, dsy};
        h->fx_ok = true;
      }
    }
    char* b;
    if ((rc = dev_alloc(h, &b, lv.nodes * tsz))) return bail(rc);
    lv.u = b;
    if ((rc = dev_alloc(h, &b, lv.nodes * tsz))) return bail(rc);
    lv.f = b;
    CK(cudaMemset(lv.u, 0, lv.nodes * tsz));
    CK(cudaMemset(lv.f, 0, lv.nodes * tsz));
    if (l > 0) {
      if ((rc = dev_alloc(h, &b, lv.nodes * tsz))) return bail(rc);
      lv.r = b;
      if ((rc = dev_alloc(h, &b, (size_t)c.nx * c.ny * nb * lv.m * lv.m * tsz))) return bail(rc);
      lv.E = b;
      if (c.nu_kind) {
        VarData vd;
        build_var(h->mx, h->my, lv.p, c.nu_kind, c.nu_a, c.nu_b, vd);
        std::vector<double> inv(vd.nu_bar.size());
        for (size_t k = 0; k < inv.size(); ++k) inv[k] = 1.0 / vd.nu_bar[k];
        double *gx, *gy, *dd;
        float *gxf, *gyf, *ddf;
        if ((rc = upload(h, &gx, vd.Gx)) || (rc = upload(h, &gy, vd.Gy)) || (rc = upload(h, &dd, vd.D)) ||
            (rc = upload(h, &gxf, vd.Gx)) || (rc = upload(h, &gyf, vd.Gy)) || (rc = upload(h, &ddf, vd.D)) ||
            (rc = upload(h, &lv.nu_inv64, inv)) || (rc = upload(h, &lv.nu_inv32, inv)))
          return bail(rc);
        lv.var = true;
        lv.v64 = VarView<double>{gx, gy, dd, nullptr};
        lv.v32 = VarView<float>{gxf, gyf, ddf, nullptr};
        // the element products reuse the level's correction buffer (n_e m^2 >= n_e (p+1)^2)
        if (h->mixed) lv.v32.E = static_cast<float*>(lv.E);
        else lv.v64.E = static_cast<double*>(lv.E);
        if (l == L && h->mixed) {  // FP64 operator of the outer MGCG on the finest level
          double* e64;
          if ((rc = dev_alloc(h, &e64, (size_t)c.nx * c.ny * (lv.p + 1) * (lv.p + 1)))) return bail(rc);
          lv.v64.E = e64;
        }
      }
    }
  }
  // coarse factors
  {
    Coarse1D cx, cy;
    std::string err = build_coarse(h->mx, cx);
    if (err.empty()) err = build_coarse(my1, cy);
    if (!err.empty()) {
      sem_destroy(h);
      return fail(SEM_BAD_ARG, err);
    }
    CoarseView& cv = h->coarse;
    cv.nux = cx.nu;
    cv.nuy = cy.nu;
    cv.firstx = cx.first;
    cv.firsty = cy.first;
    cv.Nx = h->lev[0].Nx;
    cv.Ny = h->lev[0].Ny;
    cv.periodic = c.periodic ? 1 : 0;
    cv.batch = nb;
    cv.block_rows = c.ny;  // coarse (p = 1) node rows per stacked problem
    double *Sx, *Sy, *lx, *ly, *ccx, *ccy, *T1, *T2;
    if ((rc = upload(h, &Sx, cx.S)) || (rc = upload(h, &Sy, cy.S)) || (rc = upload(h, &lx, cx.lam)) ||
        (rc = upload(h, &ly, cy.lam)) || (rc = upload(h, &ccx, cx.c)) || (rc = upload(h, &ccy, cy.c)) ||
        (rc = dev_alloc(h, &T1, (size_t)cx.nu * cy.nu * nb)) || (rc = dev_alloc(h, &T2, (size_t)cx.nu * cy.nu * nb)))
      return bail(rc);
    cv.T1 = T1;
    cv.Sx = Sx;
    cv.Sy = Sy;
    cv.lx = lx;
    cv.ly = ly;
    cv.cx = ccx;
    cv.cy = ccy;
    cv.T2 = T2;
    float *Sx32, *Sy32, *lx32, *ly32, *cx32, *cy32;
    if ((rc = upload(h, &Sx32, cx.S)) || (rc = upload(h, &Sy32, cy.S)) || (rc = upload(h, &lx32, cx.lam)) ||
        (rc = upload(h, &ly32, cy.lam)) || (rc = upload(h, &cx32, cx.c)) || (rc = upload(h, &cy32, cy.c)))
      return bail(rc);
    cv.Sx32 = Sx32;
    cv.Sy32 = Sy32;
    cv.lx32 = lx32;
    cv.ly32 = ly32;
    cv.cx32 = cx32;
    cv.cy32 = cy32;
  }
  if (c.nu_kind) {
    std::vector<double> inv;
    std::string err = coarse_var_inverse(h->mx, h->my, c.nu_kind, c.nu_a, c.nu_b, inv);
    if (!err.empty()) {
      sem_destroy(h);
      return fail(SEM_BAD_ARG, err);
    }
    if ((rc = upload(h, &h->Binv, inv))) return bail(rc);
  }
  // the persistent low-level cycle: mixed tensor-core V-cycle of the Poisson
  // operator with one pre-smoothing step and none after on levels 1 .. top
  // (p_top = min(p / 2, 8), windows m <= 16), coarse grid of at most 64 x 64
  // unknowns per problem
  if (h->mixed && h->sweep_mode != 0 && L >= 2 && !c.nu_kind && h->coarse.nux <= 64 && h->coarse.nuy <= 64) {
    const int top_l = std::min(L - 1, 3);
    bool ok = true;
    for (int l = 1; l <= top_l; ++l)
      ok = ok && h->lev[l].m <= 16 && h->ns1[l] == 1 && h->ns2[l] == 0;
    if (ok) {
      LowCycle& lc = h->lowc;
      lc.top = top_l;
      for (int l = 0; l <= top_l; ++l) {
        Level& lv = h->lev[l];
        lc.lev[l] = LowLevel{lv.x32, lv.y32, lv.J32, static_cast<float*>(lv.u), static_cast<float*>(lv.f),
                             static_cast<float*>(lv.r), static_cast<float*>(lv.E)};
      }
      lc.coarse = h->coarse;
      if ((rc = dev_alloc(h, &lc.cw, (size_t)std::max(1, nb) * 64 * 64)) || (rc = dev_alloc(h, &lc.bar, 2)))
        return bail(rc);
      CK(cudaMemset(lc.bar, 0, 2 * sizeof(unsigned)));
      lc.err = h->tc_err;
      h->low_ok = true;  // off until sem_set_low_cycle or sem_autotune turns it on
    }
  }
  // MGCG vectors, partial sums, per-iteration scalars
  h->n = top(h).nodes;
  h->rows_top = c.ny * c.p;
  h->n_unknowns = (long)nb * (long)(c.periodic ? c.nx * c.p : c.nx * c.p - 1) *
                  (long)(c.periodic ? c.ny * c.p : c.ny * c.p - 1);
  double** vecs[] = {&h->u, &h->r, &h->p, &h->q, &h->z, &h->r_old, &h->fi};
  for (double** v : vecs) {
    if ((rc = dev_alloc(h, v, h->n))) return bail(rc);
    CK(cudaMemset(*v, 0, h->n * sizeof(double)));
  }
  if ((rc = dev_alloc(h, &h->part, 4 * kMaxPartials))) return bail(rc);
  const int ni = c.i_max + 2;
  const size_t nsc = (size_t)5 * ni * nb + nb;
  double* sc;
  if ((rc = dev_alloc(h, &sc, nsc))) return bail(rc);
  CK(cudaMemset(sc, 0, nsc * sizeof(double)));
  h->st.nb = nb;
  h->st.stride = ni;
  h->st.seg_len = nb > 1 ? (long)h->rows_top * top(h).Nx : h->n;
  h->st.alpha = sc;
  h->st.beta = sc + (size_t)ni * nb;
  h->st.delta = sc + (size_t)2 * ni * nb;
  h->st.pq = sc + (size_t)3 * ni * nb;
  h->st.rr = sc + (size_t)4 * ni * nb;
  h->st.rmax = sc + (size_t)5 * ni * nb;
  int* fl;
  const size_t nfl = (size_t)3 * nb + 4;
  if ((rc = dev_alloc(h, &fl, nfl))) return bail(rc);
  CK(cudaMemset(fl, 0, nfl * sizeof(int)));
  h->st.flags = fl;                 // [nb][2]
  h->st.iters = fl + 2 * nb;        // [nb]
  h->st.iter = fl + 3 * nb;         // [2]
  h->st.ticket = reinterpret_cast<unsigned*>(fl + 3 * nb + 2);
  h->st.active = fl + 3 * nb + 3;
  if (cudaMallocHost(&h->flags_host, 2 * sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    h->flags_host = nullptr;
    sem_destroy(h);
    return fail(SEM_OOM, "cudaMallocHost failed");
  }
  CK(cudaDeviceSynchronize());
  *out = h;
  return SEM_OK;
}

// (s, kt) of every interface line and level from the weight network: the
// features of sem_learned_features, one forward pass (with the output
// transform) on the current device, widened to double.  lx / ly receive the
// layout of sem_config.learned_x / learned_y.
static int learned_from_network(const sem_config& c, const float* params, std::vector<double>& lx,
                                std::vector<double>& ly) {
  sem_config cw = c;
  cw.weight = SEM_W_QUINTIC;
  cw.learned_x = cw.learned_y = nullptr;
  int L, rc;
  if ((rc = validate(cw, L))) return rc;
  const size_t nfx = (size_t)(L + 1) * (c.nx + 1), nfy = (size_t)(L + 1) * (c.ny + 1);
  std::vector<float> fx(4 * nfx), fy(4 * nfy);
  if ((rc = sem_learned_features(&cw, fx.data(), fy.data()))) return rc;
  const size_t nmax = std::max(nfx, nfy);
  float *dp = nullptr, *dX = nullptr, *dY = nullptr;
  auto cleanup = [&]() {
    cudaFree(dp);
    cudaFree(dX);
    cudaFree(dY);
  };
  if (cudaMalloc(&dp, SEM_MLP_PARAMS * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&dX, 4 * nmax * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&dY, 2 * nmax * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(SEM_OOM, "weight network: cudaMalloc failed");
  }
  std::vector<float> y;
  for (int dir = 0; dir < 2 && rc == SEM_OK; ++dir) {
    const std::vector<float>& f = dir ? fy : fx;
    const size_t n = dir ? nfy : nfx;
    y.assign(2 * n, 0.f);
    if (cudaMemcpy(dp, params, SEM_MLP_PARAMS * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(dX, f.data(), 4 * n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      rc = fail(SEM_CUDA_ERROR, "weight network: upload failed");
      break;
    }
    if ((rc = sem_mlp_forward(dp, dX, (int32_t)n, dY, 1, nullptr))) break;
    if (cudaMemcpy(y.data(), dY, 2 * n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      rc = fail(SEM_CUDA_ERROR, "weight network: forward pass failed");
      break;
    }
    std::vector<double>& out = dir ? ly : lx;
    out.assign(y.begin(), y.end());
  }
  cleanup();
  return rc;
}

int sem_create(const sem_config* cfg, sem_handle** out) {
  g_err.clear();
  if (!cfg || !out) return fail(SEM_BAD_ARG, "null argument");
  if (cfg->weight == SEM_W_LEARNED && !cfg->learned_x && !cfg->learned_y && cfg->mlp_params) {
    std::vector<double> lx, ly;
    int rc = learned_from_network(*cfg, cfg->mlp_params, lx, ly);
    if (rc) return rc;
    sem_config c = *cfg;
    c.learned_x = lx.data();
    c.learned_y = ly.data();
    return create_handle(c, 1, out);
  }
  return create_handle(*cfg, 1, out);
}

int sem_mlp_load(sem_handle* h, const float* params) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!params) return fail(SEM_BAD_ARG, "null parameters");
  if (h->nb != 1) return fail(SEM_BAD_ARG, "sem_mlp_load: not for a handle of stacked problems");
  if (cudaSetDevice(h->device) != cudaSuccess) {
    cudaGetLastError();
    return fail(SEM_CUDA_ERROR, "cannot make the handle's device current");
  }
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return fail(SEM_CUDA_ERROR, "device error before sem_mlp_load");
  }
  sem_config c = h->cfg;
  const std::vector<double> xe = h->mx.edges, ye = h->my.edges;  // the handle's own mesh
  c.x_edges = xe.data();
  c.y_edges = ye.data();
  c.weight = SEM_W_LEARNED;
  c.learned_x = c.learned_y = nullptr;
  std::vector<double> lx, ly;
  if ((rc = learned_from_network(c, params, lx, ly))) return rc;
  c.learned_x = lx.data();
  c.learned_y = ly.data();
  sem_handle* fresh = nullptr;
  if ((rc = create_handle(c, 1, &fresh))) return rc;
  std::swap(*h, *fresh);  // h takes the new state; fresh now owns the old one
  sem_destroy(fresh);
  return SEM_OK;
}

int sem_sizes(const sem_handle* h, int64_t* n_unknowns, int64_t* nx_nodes, int64_t* ny_nodes) {
  if (!h) return fail(SEM_BAD_ARG, "null handle");
  if (n_unknowns) *n_unknowns = h->n_unknowns;
  if (nx_nodes) *nx_nodes = top(h).Nx;
  if (ny_nodes) *ny_nodes = top(h).Ny;
  return SEM_OK;
}

int sem_coords(const sem_handle* h, double* x, double* y) {
  if (!h) return fail(SEM_BAD_ARG, "null handle");
  if (x) std::memcpy(x, h->xc.data(), h->xc.size() * sizeof(double));
  if (y) std::memcpy(y, h->yc.data(), h->yc.size() * sizeof(double));
  return SEM_OK;
}

int sem_mass(sem_handle* h, const double* f, double* b, void* stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!f || !b) return fail(SEM_BAD_ARG, "null vector");
  cudaStream_t s = as_stream(stream);
  int np = 0;
  KL(h, SEM_K_VECTOR, s, launch_mass(top(h).x64, top(h).y64, f, b, h->part, &np, s));
  if (h->cfg.periodic) KL(h, SEM_K_VECTOR, s, launch_sub_mean(h->n, b, h->part, np, s));
  return SEM_OK;
}

int sem_apply(sem_handle* h, const double* u, double* Au, void* stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!u || !Au) return fail(SEM_BAD_ARG, "null vector");
  return apply64(h, u, nullptr, Au, 0, nullptr, as_stream(stream));
}

int sem_smooth(sem_handle* h, double* u, const double* f, int32_t n_it, void* stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!u || !f || n_it < 0) return fail(SEM_BAD_ARG, "invalid argument");
  cudaStream_t s = as_stream(stream);
  const Level& lv = top(h);
  if (h->mult)  // Alg. 1: every local solve forms its own residual
    return h->mixed ? mult_sweeps<float, double, double>(h, lv, f, u, n_it, s)
                    : mult_sweeps<double, double, double>(h, lv, f, u, n_it, s);
  for (int k = 0; k < n_it; ++k) {
    if ((rc = apply64(h, u, f, h->r, 0, nullptr, s))) return rc;
    rc = h->mixed ? sweep<float, double, double>(h, lv, h->r, u, true, s)
                  : sweep<double, double, double>(h, lv, h->r, u, true, s);
    if (rc) return rc;
  }
  return SEM_OK;
}

int sem_vcycle(sem_handle* h, double* u, const double* f, void* stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!u || !f) return fail(SEM_BAD_ARG, "null vector");
  cudaStream_t s = as_stream(stream);
  // MultigridCycle(u, f) = u + MultigridCycle(0, f - A u): the cycle is affine
  if ((rc = apply64(h, u, f, h->r, 0, nullptr, s))) return rc;
  if ((rc = precond(h, h->r, h->z, s))) return rc;
  KL(h, SEM_K_VECTOR, s, launch_axpy(h->n, 1.0, h->z, u, s));
  return SEM_OK;
}

int sem_mg_solve(sem_handle* h, double* u, const double* f, sem_result* res, double* history, int32_t hlen,
                 void* stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!u || !f || !res) return fail(SEM_BAD_ARG, "null argument");
  cudaStream_t s = as_stream(stream);
  std::vector<double> part(kMaxPartials);
  auto norm = [&](double& out) -> int {
    int np = 0;
    if ((rc = apply64(h, u, f, h->r, 2, &np, s))) return rc;
    CK(cudaMemcpyAsync(part.data(), h->part, np * sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    double a = 0.0;
    for (int i = 0; i < np; ++i) a += part[i];
    out = std::sqrt(a);
    return SEM_OK;
  };
  double r0, rn;
  if ((rc = norm(r0))) return rc;
  if (history && hlen > 0) history[0] = r0;
  rn = r0;
  int it = 0;
  int status = SEM_NOT_CONVERGED;
  if (!(r0 > 0)) status = std::isfinite(r0) ? SEM_OK : SEM_BREAKDOWN;
  while (status == SEM_NOT_CONVERGED && it < h->cfg.i_max) {
    if ((rc = precond(h, h->r, h->z, s))) return rc;
    KL(h, SEM_K_VECTOR, s, launch_axpy(h->n, 1.0, h->z, u, s));
    ++it;
    if ((rc = norm(rn))) return rc;
    if (history && it < hlen) history[it] = rn;
    if (!std::isfinite(rn)) status = SEM_BREAKDOWN;
    else if (rn <= h->cfg.tol * r0) status = SEM_OK;
  }
  bool timeout = false;
  if ((rc = take_tc_err(h, s, timeout))) return rc;
  if (timeout) status = SEM_TIMEOUT;
  res->iterations = it;
  res->status = status;
  res->res0 = r0;
  res->res = rn;
  res->rbar = (it > 0 && rn > 0) ? std::log10(r0 / rn) / it : 0.0;
  return status;
}

// run the MGCG of all problems of h on the vectors already in h->u / h->fi:
// launch by launch on the first solve (and with profiling on), afterwards by
// replaying the captured graph
static int run_solve(sem_handle* h, cudaStream_t s) {
  int rc;
  const bool use_graph = !h->prof && h->solves > 0;
  if (use_graph && !h->graph_exec) {
    CK(cudaStreamSynchronize(s));
    if ((rc = build_graph(h))) return rc;
  }
  if (use_graph) {
    CK(cudaGraphLaunch(h->graph_exec, s));
  } else {
    if ((rc = pcg_prologue(h, s, 0, 0))) return rc;
    for (;;) {
      if ((rc = sync_flags(h, s))) return rc;
      if (h->flags_host[0] == 0) break;
      if ((rc = pcg_body(h, s, 0, 0))) return rc;
    }
  }
  return SEM_OK;
}

// per-problem results after a solve (sync); launches of a replayed graph are
// added to the tracing counters
static int collect(sem_handle* h, cudaStream_t s, bool graph_used, sem_result* res, double* const* hist, int hlen) {
  const int nb = h->nb, stride = h->st.stride;
  std::vector<int> fl(3 * nb);
  CK(cudaMemcpyAsync(fl.data(), h->st.flags, 3 * nb * sizeof(int), cudaMemcpyDeviceToHost, s));
  std::vector<double> rr((size_t)nb * stride);
  CK(cudaMemcpyAsync(rr.data(), h->st.rr, rr.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  bool timeout = false;
  int rc0 = take_tc_err(h, s, timeout);
  if (rc0) return rc0;
  int itmax = 0;
  for (int k = 0; k < nb; ++k) {
    const int it = fl[2 * nb + k];
    itmax = std::max(itmax, it);
    const double* r = rr.data() + (size_t)k * stride;
    res[k].iterations = it;
    res[k].status = fl[2 * k + 1];
    res[k].res0 = std::sqrt(r[0]);
    res[k].res = std::sqrt(r[it]);
    res[k].rbar = (it > 0 && r[it] > 0) ? std::log10(std::sqrt(r[0] / r[it])) / it : 0.0;
    if (timeout) res[k].status = SEM_TIMEOUT;
    if (hist && hist[k])
      for (int i = 0; i <= it && i < hlen; ++i) hist[k][i] = std::sqrt(r[i]);
  }
  if (graph_used)
    for (int c = 0; c < SEM_K_NCLASS; ++c)
      h->launches[c] += h->graph_pro[c] + (long long)std::max(0, itmax - 1) * h->graph_body[c];
  h->solves++;
  return SEM_OK;
}

int sem_pcg_solve(sem_handle* h, double* u, const double* f, sem_result* res, double* history, int32_t hlen,
                  void* stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!u || !f || !res) return fail(SEM_BAD_ARG, "null argument");
  if (h->nb != 1) return fail(SEM_BAD_ARG, "use sem_batch_solve for stacked problems");
  cudaStream_t s = as_stream(stream);
  const int rows = top(h).Ny - 1, Nx = top(h).Nx;
  if (!h->cfg.periodic) {
    KL(h, SEM_K_VECTOR, s, launch_stack_in(nullptr, f, h->fi, 1, rows, Nx, h->n, s));
    KL(h, SEM_K_VECTOR, s, launch_stack_in(nullptr, u, h->u, 1, rows, Nx, h->n, s));
  } else {
    CK(cudaMemcpyAsync(h->fi, f, h->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK(cudaMemcpyAsync(h->u, u, h->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  }
  const bool graph_used = !h->prof && h->solves > 0;
  if ((rc = run_solve(h, s))) return rc;
  CK(cudaMemcpyAsync(u, h->u, h->n * sizeof(double), cudaMemcpyDeviceToDevice, s));
  double* hp[1] = {history};
  if ((rc = collect(h, s, graph_used, res, hp, hlen))) return rc;
  return res->status;
}

int sem_profile(sem_handle* h, int32_t enable) {
  int rc = check_handle(h);
  if (rc) return rc;
  for (auto& c : h->launches) c = 0;
  h->ev_used = 0;
  h->prof = enable != 0;
  return SEM_OK;
}

int sem_autotune(sem_handle* h, const char* cache_path, void* stream) {
  int rc = check_handle(h);
  if (rc) return rc;
  return autotune(h, cache_path ? std::string(cache_path) : std::string(), as_stream(stream));
}

int sem_set_low_cycle(sem_handle* h, int32_t enable) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (enable != 0 && enable != 1) return fail(SEM_BAD_ARG, "enable must be 0 or 1");
  if (enable && !h->low_ok) return fail(SEM_BAD_ARG, "no persistent low-level cycle for this configuration");
  CK(cudaDeviceSynchronize());
  h->low_on = enable != 0;
  drop_graph(h);
  return SEM_OK;
}

int sem_set_fixed_point_operator(sem_handle* h, int32_t enable) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (enable != 0 && enable != 1) return fail(SEM_BAD_ARG, "enable must be 0 or 1");
  if (enable && !h->fx_ok) return fail(SEM_BAD_ARG, "no fixed-point operator for this configuration");
  CK(cudaDeviceSynchronize());
  h->fx_on = enable != 0;
  drop_graph(h);
  return SEM_OK;
}

int sem_get_fixed_point_operator(const sem_handle* h, int32_t* available, int32_t* enabled) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (available) *available = h->fx_ok ? 1 : 0;
  if (enabled) *enabled = (h->fx_ok && h->fx_on) ? 1 : 0;
  return SEM_OK;
}

int sem_set_fused_prolongation(sem_handle* h, int32_t enable) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (enable != 0 && enable != 1) return fail(SEM_BAD_ARG, "enable must be 0 or 1");
  if (enable && !h->chain_ok) return fail(SEM_BAD_ARG, "no fused prolongation for this configuration");
  CK(cudaDeviceSynchronize());
  h->chain_on = enable != 0;
  drop_graph(h);
  return SEM_OK;
}

int sem_get_fused_prolongation(const sem_handle* h, int32_t* available, int32_t* enabled) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (available) *available = h->chain_ok ? 1 : 0;
  if (enabled) *enabled = (h->chain_ok && h->chain_on) ? 1 : 0;
  return SEM_OK;
}

int sem_get_low_cycle(const sem_handle* h, int32_t* available, int32_t* enabled) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (available) *available = h->low_ok ? 1 : 0;
  if (enabled) *enabled = (h->low_ok && h->low_on) ? 1 : 0;
  return SEM_OK;
}

int sem_get_tune(const sem_handle* h, int32_t level, sem_level_tune* t) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!t) return fail(SEM_BAD_ARG, "null argument");
  if (level < 1 || level > h->L) return fail(SEM_BAD_ARG, "level must be in 1..log2(p)");
  const TuneVal& v = h->lev[level].tune;
  t->fuse = v.fuse;
  t->spw = v.spw;
  t->tc = v.tc;
  t->tc_available = h->lev[level].tc.ngroups > 0;
  t->eo = v.eo;
  t->us = v.us;
  return SEM_OK;
}

int sem_set_tune(sem_handle* h, int32_t level, const sem_level_tune* t) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (!t) return fail(SEM_BAD_ARG, "null argument");
  if (level < 1 || level > h->L) return fail(SEM_BAD_ARG, "level must be in 1..log2(p)");
  if (t->fuse < 0 || t->fuse > 1 || t->spw < 1 || t->spw > 64 || t->tc < 0 || t->tc > 1 || t->eo < -1 || t->eo > 1)
    return fail(SEM_BAD_ARG, "need fuse, tc in {0, 1}, eo in {-1, 0, 1}, 1 <= spw <= 64");
  if (t->tc && h->lev[level].tc.ngroups == 0) return fail(SEM_BAD_ARG, "no tcgen05 sweep on this level");
  CK(cudaDeviceSynchronize());
  TuneVal& v = h->lev[level].tune;
  v.fuse = t->fuse;
  v.spw = t->spw;
  v.tc = t->tc;
  v.eo = t->eo;
  v.us = t->us;
  drop_graph(h);
  return SEM_OK;
}

int sem_profile_read(sem_handle* h, double* ms, int64_t* launches) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (ms)
    for (int c = 0; c < SEM_K_NCLASS; ++c) ms[c] = 0.0;
  for (int k = 0; k < h->ev_used; ++k) {
    CK(cudaEventSynchronize(h->ev[2 * k + 1]));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, h->ev[2 * k], h->ev[2 * k + 1]));
    if (ms) ms[h->ev_cls[k]] += t;
  }
  if (launches)
    for (int c = 0; c < SEM_K_NCLASS; ++c) launches[c] = h->launches[c];
  return SEM_OK;
}

int sem_profile_read_level(sem_handle* h, int32_t level, double* ms, int64_t* launches) {
  int rc = check_handle(h);
  if (rc) return rc;
  if (level < -1 || level > h->L) return fail(SEM_BAD_ARG, "level must be in [-1, L]");
  for (int c = 0; c < SEM_K_NCLASS; ++c) {
    if (ms) ms[c] = 0.0;
    if (launches) launches[c] = 0;
  }
  for (int k = 0; k < h->ev_used; ++k) {
    if (h->ev_lvl[k] != level) continue;
    CK(cudaEventSynchronize(h->ev[2 * k + 1]));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, h->ev[2 * k], h->ev[2 * k + 1]));
    if (ms) ms[h->ev_cls[k]] += t;
    if (launches) launches[h->ev_cls[k]] += h->ev_nk[k];
  }
  return SEM_OK;
}

}  // extern "C"

// ---- batched solves: many independent problems, one graph launch ---------

namespace {

struct BatchGroup {
  sem_handle* h = nullptr;
  std::vector<int> members;  // problem indices in the caller's order
  cudaStream_t branch = nullptr, body = nullptr;
};

bool same_group(const sem_config& a, const sem_config& b) {
  return a.nx == b.nx && a.ny == b.ny && a.p == b.p && a.periodic == b.periodic && a.lx == b.lx && a.ly == b.ly &&
         a.overlap_rule == b.overlap_rule && a.overlap == b.overlap && a.weight == b.weight && a.ns1 == b.ns1 &&
         a.ns2 == b.ns2 && a.variable_cycle == b.variable_cycle && a.precision == b.precision && a.tol == b.tol &&
         a.i_max == b.i_max && a.nu_kind == b.nu_kind && a.nu_a == b.nu_a && a.nu_b == b.nu_b;
}

// the finest-level operator tiles (tile_elems(p) elements high) must not straddle two
// stacked problems: their partial sums are per problem
bool tiles_fit(const sem_config& c) { return c.ny % tile_elems(c.p) == 0; }

bool stackable(const sem_config& c) {
  return !c.periodic && !c.x_edges && !c.y_edges && !c.nu_kind && c.weight != SEM_W_LEARNED && tiles_fit(c);
}

}  // namespace

struct sem_batch {
  int n = 0;
  int device = 0;
  std::vector<BatchGroup> groups;
  const double** host_ptrs = nullptr;  // pinned: [f pointers | u pointers] in group-member order
  const double** dev_ptrs = nullptr;   // device copy of host_ptrs
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t main = nullptr;
  int solves = 0;
};

extern "C" {

void sem_batch_destroy(sem_batch* b) {
  if (!b) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  cudaDeviceSynchronize();
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->main) cudaStreamDestroy(b->main);
  for (auto& g : b->groups) {
    if (g.branch) cudaStreamDestroy(g.branch);
    if (g.body) cudaStreamDestroy(g.body);
    sem_destroy(g.h);
  }
  if (b->dev_ptrs) cudaFree(b->dev_ptrs);
  if (b->host_ptrs) cudaFreeHost(b->host_ptrs);
  if (prev >= 0) cudaSetDevice(prev);
  cudaGetLastError();
  delete b;
}

int sem_batch_create(const sem_config* cfgs, int32_t n, sem_batch** out) {
  g_err.clear();
  if (!cfgs || !out || n < 1) return fail(SEM_BAD_ARG, "invalid argument");
  sem_batch* b = new sem_batch();
  b->n = n;
  if (cudaGetDevice(&b->device) != cudaSuccess) {
    cudaGetLastError();
    delete b;
    return fail(SEM_CUDA_ERROR, "no usable CUDA device");
  }
  // group identical stackable configurations; anything else solves alone
  std::vector<std::vector<int>> groups;
  for (int k = 0; k < n; ++k) {
    if (cfgs[k].periodic) {
      delete b;
      return fail(SEM_BAD_ARG, "batched problems need Dirichlet walls");
    }
    int found = -1;
    if (stackable(cfgs[k]))
      for (size_t g = 0; g < groups.size(); ++g)
        if (stackable(cfgs[groups[g][0]]) && same_group(cfgs[groups[g][0]], cfgs[k]) &&
            (long)(groups[g].size() + 1) * cfgs[k].ny <= 4096) {
          found = (int)g;
          break;
        }
    if (found < 0) {
      groups.push_back({k});
    } else {
      groups[found].push_back(k);
    }
  }
  for (auto& mem : groups) {
    BatchGroup g;
    g.members = mem;
    int rc = create_handle(cfgs[mem[0]], (int)mem.size(), &g.h);
    if (rc) {
      sem_batch_destroy(b);
      return rc;
    }
    b->groups.push_back(g);
  }
  if (cudaMallocHost(&b->host_ptrs, 2 * n * sizeof(double*)) != cudaSuccess ||
      cudaMalloc(&b->dev_ptrs, 2 * n * sizeof(double*)) != cudaSuccess) {
    cudaGetLastError();
    sem_batch_destroy(b);
    return fail(SEM_OOM, "pointer tables");
  }
  // groups run as concurrent branches of one graph: a grid-wide cooperative
  // kernel per group could not be resident together, so with several groups
  // the low levels stay on per-level launches
  if (b->groups.size() > 1)
    for (auto& g : b->groups) g.h->low_ok = g.h->low_on = false;
  *out = b;
  return SEM_OK;
}

int sem_batch_info(const sem_batch* b, int32_t* groups, int64_t* unknowns) {
  if (!b) return fail(SEM_BAD_ARG, "null batch");
  if (groups) *groups = (int32_t)b->groups.size();
  if (unknowns) {
    int64_t t = 0;
    for (auto& g : b->groups) t += g.h->n_unknowns;
    *unknowns = t;
  }
  return SEM_OK;
}

int sem_batch_solve(sem_batch* b, double* const* u, const double* const* f, sem_result* res, void* stream) {
  if (!b || !u || !f || !res) return fail(SEM_BAD_ARG, "null argument");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) {
    cudaGetLastError();
    return fail(SEM_BAD_ARG, "the current CUDA device is not the batch's device");
  }
  cudaStream_t s = as_stream(stream);
  // pointer tables: f of every member, then u, in group order
  int o = 0;
  for (auto& g : b->groups)
    for (int k : g.members) {
      if (!u[k] || !f[k]) return fail(SEM_BAD_ARG, "null vector in the batch");
      b->host_ptrs[o] = f[k];
      b->host_ptrs[b->n + o] = u[k];
      ++o;
    }
  CK(cudaMemcpyAsync(b->dev_ptrs, b->host_ptrs, 2 * b->n * sizeof(double*), cudaMemcpyHostToDevice, s));
  auto stage_in = [&](BatchGroup& g, int off, cudaStream_t st) -> int {
    sem_handle* h = g.h;
    const int rows = h->rows_top, Nx = top(h).Nx, nm = (int)g.members.size();
    KL(h, SEM_K_VECTOR, st, launch_stack_in(b->dev_ptrs + off, nullptr, h->fi, nm, rows, Nx, h->st.seg_len, st));
    KL(h, SEM_K_VECTOR, st,
       launch_stack_in(b->dev_ptrs + b->n + off, nullptr, h->u, nm, rows, Nx, h->st.seg_len, st));
    return SEM_OK;
  };
  auto stage_out = [&](BatchGroup& g, int off, cudaStream_t st) -> int {
    sem_handle* h = g.h;
    const int rows = h->rows_top, Nx = top(h).Nx, nm = (int)g.members.size();
    KL(h, SEM_K_VECTOR, st,
       launch_stack_out(h->u, const_cast<double* const*>(b->dev_ptrs + b->n + off), nullptr, nm, rows, Nx,
                        h->st.seg_len, st));
    return SEM_OK;
  };
  int rc;
  const bool graph_used = b->solves > 0;
  if (!graph_used) {
    // first solve: group by group, launch by launch (loads modules, sets limits)
    int off = 0;
    for (auto& g : b->groups) {
      if ((rc = stage_in(g, off, s)) || (rc = run_solve(g.h, s)) || (rc = stage_out(g, off, s))) return rc;
      off += (int)g.members.size();
    }
  } else {
    if (!b->exec) {
      // every group becomes one branch of a single graph: stage in, prologue,
      // WHILE node over the MGCG iteration, stage out
      CK(cudaStreamSynchronize(s));
      CK(cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking));
      for (auto& g : b->groups) {
        CK(cudaStreamCreateWithFlags(&g.branch, cudaStreamNonBlocking));
        CK(cudaStreamCreateWithFlags(&g.body, cudaStreamNonBlocking));
      }
      cudaEvent_t fork;
      CK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
      CK(cudaStreamBeginCapture(b->main, cudaStreamCaptureModeRelaxed));
      CK(cudaEventRecord(fork, b->main));
      int off = 0;
      std::vector<cudaEvent_t> joins;
      for (auto& g : b->groups) {
        cudaEvent_t join;
        CK(cudaEventCreateWithFlags(&join, cudaEventDisableTiming));
        joins.push_back(join);
        CK(cudaStreamWaitEvent(g.branch, fork, 0));
        if ((rc = stage_in(g, off, g.branch)) || (rc = capture_solve(g.h, g.branch, g.body)) ||
            (rc = stage_out(g, off, g.branch))) {
          end_capture_discard(b->main);
          return rc;
        }
        CK(cudaEventRecord(join, g.branch));
        CK(cudaStreamWaitEvent(b->main, join, 0));
        off += (int)g.members.size();
      }
      CK(cudaStreamEndCapture(b->main, &b->graph));
      CK(cudaGraphInstantiate(&b->exec, b->graph, 0));
      CK(cudaEventDestroy(fork));
      for (auto e : joins) CK(cudaEventDestroy(e));
      for (auto& g : b->groups) g.h->launches[SEM_K_VECTOR] -= 3;  // staging launches counted at replay below
    }
    CK(cudaGraphLaunch(b->exec, s));
    for (auto& g : b->groups) g.h->launches[SEM_K_VECTOR] += 3;
  }
  // results, problem by problem
  for (auto& g : b->groups) {
    std::vector<sem_result> r(g.members.size());
    if ((rc = collect(g.h, s, graph_used, r.data(), nullptr, 0))) return rc;
    for (size_t j = 0; j < g.members.size(); ++j) res[g.members[j]] = r[j];
  }
  b->solves++;
  int worst = SEM_OK;
  for (int k = 0; k < b->n; ++k) worst = std::max(worst, (int)res[k].status);
  return worst;
}

int sem_batch_autotune(sem_batch* b, const char* cache_path, void* stream) {
  if (!b) return fail(SEM_BAD_ARG, "null batch");
  for (auto& g : b->groups) {
    int rc = sem_autotune(g.h, cache_path, stream);
    if (rc) return rc;
  }
  // the batch graph holds the old launch shapes: capture a new one next solve
  CK(cudaDeviceSynchronize());
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->main) cudaStreamDestroy(b->main);
  b->exec = nullptr;
  b->graph = nullptr;
  b->main = nullptr;
  for (auto& g : b->groups) {
    if (g.branch) cudaStreamDestroy(g.branch);
    if (g.body) cudaStreamDestroy(g.body);
    g.branch = g.body = nullptr;
  }
  return SEM_OK;
}

int sem_batch_launches(const sem_batch* b, int64_t* launches) {
  if (!b || !launches) return fail(SEM_BAD_ARG, "null argument");
  *launches = 0;
  for (auto& g : b->groups)
    for (int c = 0; c < SEM_K_NCLASS; ++c) *launches += g.h->launches[c];
  return SEM_OK;
}

}  // extern "C"

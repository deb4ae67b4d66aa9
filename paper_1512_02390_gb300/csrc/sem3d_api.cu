// C ABI of the three-dimensional extension (include/sem_schwarz3d.h).
//
// A handle holds the levels p_l = 2^l of Alg. 3 with the 1D tables of every
// direction (the same host set-up as the 2D solver: GLL set, element
// matrices, padded window factors and weights per element class, coarse
// eigenpairs), the level vectors in the V-cycle's type, and the FP64 vectors
// of Alg. 4.  The MGCG iteration is driven by the host, which reads the dot
// products of every iteration; every vector operation runs in the kernels of
// k_3d.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "kernels3d.h"
#include "sem_schwarz3d.h"
#include "setup.h"

namespace sem {
void set_last_error(const std::string& msg);  // sem_api.cu
}

using namespace sem;

namespace {

int fail3(int code, const std::string& m) {
  set_last_error(m);
  return code;
}

#define CK3(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      cudaGetLastError();                                                                      \
      return fail3(SEM_CUDA_ERROR, std::string(#call) + ": " + cudaGetErrorString(e_));        \
    }                                                                                          \
  } while (0)

struct Level3 {
  int p = 0, n_o = 0, m = 0;
  long nodes = 0;
  Dir3<double> d64{};
  Dir3<float> d32{};
  double* J64 = nullptr;  // interpolation from level l-1 to l
  float* J32 = nullptr;
  void* u = nullptr;      // level vectors in the V-cycle type
  void* f = nullptr;
  void* r = nullptr;
  void* E = nullptr;      // n_e m^3 Schwarz corrections
  void* Ec = nullptr;     // n_e (p/2 + 1)^3 element restrictions
};

}  // namespace

struct sem3_handle {
  sem3_config cfg{};
  int device = 0, L = 0;
  bool mixed = false;
  std::vector<Level3> lev;
  Coarse3<double> c64{};
  Coarse3<float> c32{};
  void *cw1 = nullptr, *cw2 = nullptr;
  long n = 0, n_unknowns = 0;
  double *r = nullptr, *p = nullptr, *q = nullptr, *z = nullptr, *r_old = nullptr, *ones = nullptr;
  double* part = nullptr;
  std::vector<double> coords[3];
  std::vector<void*> allocs;
};

namespace {

template <typename T>
int alloc3(sem3_handle* h, T** ptr, size_t count) {
  void* d = nullptr;
  if (cudaMalloc(&d, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return fail3(SEM_OOM, "cudaMalloc failed");
  }
  h->allocs.push_back(d);
  *ptr = static_cast<T*>(d);
  return SEM_OK;
}

template <typename T, typename S>
int upload3(sem3_handle* h, T** ptr, const std::vector<S>& v) {
  std::vector<T> tmp(v.begin(), v.end());
  int rc = alloc3(h, ptr, tmp.size());
  if (rc) return rc;
  CK3(cudaMemcpy(*ptr, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice));
  return SEM_OK;
}

template <typename T>
int upload_view(sem3_handle* h, const Dir1D& d, DirView<T>& v) {
  v.p = d.p;
  v.n = d.n;
  v.N = d.N;
  v.periodic = d.periodic ? 1 : 0;
  v.n_o = d.n_o;
  v.m = d.m;
  v.segN = 0;
  std::vector<double> S, lam, w;
  for (const auto& t : d.tables) {
    S.insert(S.end(), t.S.begin(), t.S.end());
    lam.insert(lam.end(), t.lam.begin(), t.lam.end());
    w.insert(w.end(), t.w.begin(), t.w.end());
  }
  T *Le, *Mg, *Sd, *ld, *wd;
  int* tab;
  int rc;
  if ((rc = upload3(h, &Le, d.Le)) || (rc = upload3(h, &Mg, d.Mglob)) || (rc = upload3(h, &tab, d.tab)) ||
      (rc = upload3(h, &Sd, S)) || (rc = upload3(h, &ld, lam)) || (rc = upload3(h, &wd, w)))
    return rc;
  v.Le = Le;
  v.Mg = Mg;
  v.tab = tab;
  v.S = Sd;
  v.lam = ld;
  v.w = wd;
  return SEM_OK;
}

int overlap3(const sem3_config& c, int pl) {
  int n;
  switch (c.overlap_rule) {
    case SEM_OVERLAP_FIXED: n = c.overlap; break;
    case SEM_OVERLAP_FLOOR8: n = pl / 8; break;
    case SEM_OVERLAP_CEIL8: n = (pl + 7) / 8; break;
    case SEM_OVERLAP_CEIL2: n = (pl + 1) / 2; break;
    default: return -1;
  }
  return n < 0 ? -1 : std::min(n, pl - 1);
}

int validate3(const sem3_config& c, int& L) {
  L = 0;
  while ((1 << L) < c.p) ++L;
  if (c.p < 2 || c.p > 16 || (1 << L) != c.p) return fail3(SEM_BAD_ARG, "p must be a power of two in [2, 16]");
  if (c.nx < 2 || c.ny < 2 || c.nz < 2 || c.nx > 512 || c.ny > 512 || c.nz > 512)
    return fail3(SEM_BAD_ARG, "nx, ny, nz must be in [2, 512]");
  const int w = c.weight;
  if (!(w == 1 || w == 3 || w == 5 || w == 7 || w == SEM_W_TOPHAT || w == SEM_W_ARITH || w == SEM_W_IDENTITY))
    return fail3(SEM_BAD_ARG, "unknown weight function (learned weights are 2D only)");
  if (c.overlap_rule < 0 || c.overlap_rule > 3 || (c.overlap_rule == SEM_OVERLAP_FIXED && c.overlap < 0))
    return fail3(SEM_BAD_ARG, "invalid overlap rule");
  if (c.precision != SEM_PREC_FP64 && c.precision != SEM_PREC_FP32)
    return fail3(SEM_BAD_ARG, "3D: precision must be FP64 or FP32");
  if (c.ns1 < 0 || c.ns2 < 0 || c.ns1 + c.ns2 < 1 || c.ns1 > 16 || c.ns2 > 16)
    return fail3(SEM_BAD_ARG, "need 0 <= ns1, ns2 <= 16 and ns1 + ns2 >= 1");
  if (!(c.tol >= 0.0) || c.i_max < 1 || c.i_max > 100000) return fail3(SEM_BAD_ARG, "invalid tol or i_max");
  if (!(c.lx > 0) || !(c.ly > 0) || !(c.lz > 0)) return fail3(SEM_BAD_ARG, "lx, ly, lz must be positive");
  return SEM_OK;
}

Mesh1D mesh3(int n, double len, bool periodic) {
  Mesh1D m;
  m.n = n;
  m.periodic = periodic;
  m.edges.resize(n + 1);
  for (int i = 0; i <= n; ++i) m.edges[i] = len * i / n;
  return m;
}

int check3(const sem3_handle* h) {
  if (!h) return fail3(SEM_BAD_ARG, "null handle");
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != h->device) {
    cudaGetLastError();
    return fail3(SEM_BAD_ARG, "the current CUDA device is not the handle's device");
  }
  return SEM_OK;
}

template <typename T>
const Dir3<T>& D3(const Level3& l) {
  if constexpr (std::is_same<T, double>::value) return l.d64; else return l.d32;
}
template <typename T>
const T* J3(const Level3& l) {
  if constexpr (std::is_same<T, double>::value) return l.J64; else return l.J32;
}

// u = (accum ? u : 0) + n Schwarz sweeps on level l: the first from r (the
// level's right side when starting from u = 0), the others on f - A u
template <typename T>
int smooth3(sem3_handle* h, const Level3& l, const T* f, T* u, int n, bool from_zero, cudaStream_t s) {
  T* r = static_cast<T*>(l.r);
  T* E = static_cast<T*>(l.E);
  for (int k = 0; k < n; ++k) {
    if (from_zero && k == 0) {
      CK3((launch3_sweep<T, T>(D3<T>(l), f, E, u, false, s)));
      continue;
    }
    CK3((launch3_apply<T, T>(D3<T>(l), u, f, r, s)));
    CK3((launch3_sweep<T, T>(D3<T>(l), r, E, u, true, s)));
  }
  return SEM_OK;
}

// z = MultigridCycle(0, rtop), Alg. 3, with the level vectors in type T
template <typename T>
int vcycle3(sem3_handle* h, const double* rtop, double* zout, cudaStream_t s) {
  constexpr bool dbl = std::is_same<T, double>::value;
  auto& lv = h->lev;
  const int L = h->L;
  const int ns1 = h->cfg.ns1, ns2 = h->cfg.ns2;
  T* fL;
  T* uL;
  if constexpr (dbl) {
    fL = const_cast<T*>(rtop);
    uL = zout;
  } else {
    fL = static_cast<T*>(lv[L].f);
    uL = static_cast<T*>(lv[L].u);
    CK3((launch3_convert<double, float>(lv[L].nodes, rtop, fL, s)));
  }
  int rc;
  for (int l = L; l >= 1; --l) {
    T* ul = l == L ? uL : static_cast<T*>(lv[l].u);
    const T* fl = l == L ? fL : static_cast<const T*>(lv[l].f);
    if (ns1 > 0) {
      if ((rc = smooth3<T>(h, lv[l], fl, ul, ns1, true, s))) return rc;
    } else {
      CK3(cudaMemsetAsync(ul, 0, lv[l].nodes * sizeof(T), s));
    }
    T* rl = static_cast<T*>(lv[l].r);
    CK3((launch3_apply<T, T>(D3<T>(lv[l]), ul, fl, rl, s)));
    CK3((launch3_restrict<T>(D3<T>(lv[l]), D3<T>(lv[l - 1]), J3<T>(lv[l]), rl, static_cast<T*>(lv[l].Ec),
                             static_cast<T*>(lv[l - 1].f), s)));
  }
  if constexpr (dbl) {
    CK3((launch3_coarse<T>(h->c64, static_cast<T*>(h->cw1), static_cast<T*>(h->cw2), static_cast<T*>(lv[0].f),
                           static_cast<T*>(lv[0].u), s)));
  } else {
    CK3((launch3_coarse<T>(h->c32, static_cast<T*>(h->cw1), static_cast<T*>(h->cw2), static_cast<T*>(lv[0].f),
                           static_cast<T*>(lv[0].u), s)));
  }
  for (int l = 1; l <= L; ++l) {
    T* ul = l == L ? uL : static_cast<T*>(lv[l].u);
    const T* fl = l == L ? fL : static_cast<const T*>(lv[l].f);
    CK3((launch3_prolong<T, T>(D3<T>(lv[l]), D3<T>(lv[l - 1]), J3<T>(lv[l]), static_cast<const T*>(lv[l - 1].u), ul,
                               ul, s)));
    if (ns2 > 0 && (rc = smooth3<T>(h, lv[l], fl, ul, ns2, false, s))) return rc;
  }
  if constexpr (!dbl) CK3((launch3_convert<float, double>(lv[L].nodes, uL, zout, s)));
  return SEM_OK;
}

int precond3(sem3_handle* h, const double* r, double* z, cudaStream_t s) {
  return h->mixed ? vcycle3<float>(h, r, z, s) : vcycle3<double>(h, r, z, s);
}

// a . b, reduced on the host in a fixed order (sync)
int dot3(sem3_handle* h, const double* a, const double* b, double* out, cudaStream_t s) {
  int np = 0;
  CK3(launch3_dot(a, b, h->n, h->part, &np, s));
  double buf[kDot3Parts];
  CK3(cudaMemcpyAsync(buf, h->part, np * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK3(cudaStreamSynchronize(s));
  double acc = 0.0;
  for (int i = 0; i < np; ++i) acc += buf[i];
  *out = acc;
  return SEM_OK;
}

cudaStream_t st3(void* s) { return static_cast<cudaStream_t>(s); }

}  // namespace

extern "C" {

void sem3_default_config(sem3_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->nx = c->ny = c->nz = 4;
  c->p = 4;
  c->lx = c->ly = c->lz = 1.0;
  c->overlap_rule = SEM_OVERLAP_FIXED;
  c->overlap = 1;
  c->weight = SEM_W_QUINTIC;
  c->ns1 = 1;
  c->precision = SEM_PREC_FP64;
  c->tol = 1e-10;
  c->i_max = 200;
}

void sem3_destroy(sem3_handle* h) {
  if (!h) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  for (void* p : h->allocs) cudaFree(p);
  if (prev >= 0) cudaSetDevice(prev);
  cudaGetLastError();
  delete h;
}

int sem3_create(const sem3_config* cfg, sem3_handle** out) {
  if (!cfg || !out) return fail3(SEM_BAD_ARG, "null argument");
  const sem3_config c = *cfg;
  int L, rc;
  if ((rc = validate3(c, L))) return rc;
  sem3_handle* h = new sem3_handle();
  h->cfg = c;
  h->L = L;
  h->mixed = c.precision == SEM_PREC_FP32;
  auto bail = [&](int code) {
    sem3_destroy(h);
    return code;
  };
  if (cudaGetDevice(&h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail3(SEM_CUDA_ERROR, "no usable CUDA device");
  }
  const bool per = c.periodic != 0;
  const Mesh1D ms[3] = {mesh3(c.nx, c.lx, per), mesh3(c.ny, c.ly, per), mesh3(c.nz, c.lz, per)};
  // the finest window must fit one CTA's shared memory
  {
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, h->device) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return fail3(SEM_CUDA_ERROR, "cannot query the shared-memory limit");
    }
    for (int l = 1; l <= L; ++l) {
      const int pl = 1 << l, no = overlap3(c, pl), m = pl + 1 + 2 * no;
      const size_t need = h->mixed ? sweep3_smem_bytes<float>(m) : sweep3_smem_bytes<double>(m);
      if (no < 0 || need > (size_t)optin) {
        delete h;
        return fail3(SEM_BAD_ARG, "3D window m = " + std::to_string(m) + " needs " + std::to_string(need) +
                                      " bytes of shared memory per block; the device allows " + std::to_string(optin));
      }
    }
  }
  const size_t tsz = h->mixed ? sizeof(float) : sizeof(double);
  const long ne = (long)c.nx * c.ny * c.nz;
  h->lev.resize(L + 1);
  for (int l = 0; l <= L; ++l) {
    Level3& lv = h->lev[l];
    lv.p = 1 << l;
    lv.n_o = l > 0 ? overlap3(c, lv.p) : 0;
    lv.m = lv.p + 1 + 2 * lv.n_o;
    Dir1D d[3];
    for (int a = 0; a < 3; ++a) {
      const std::string err = build_dir(ms[a], lv.p, lv.n_o, l > 0 ? c.weight : SEM_W_IDENTITY, d[a]);
      if (!err.empty()) {
        sem3_destroy(h);
        return fail3(SEM_BAD_ARG, "level p=" + std::to_string(lv.p) + ": " + err);
      }
    }
    if ((rc = upload_view(h, d[0], lv.d64.x)) || (rc = upload_view(h, d[1], lv.d64.y)) ||
        (rc = upload_view(h, d[2], lv.d64.z)) || (rc = upload_view(h, d[0], lv.d32.x)) ||
        (rc = upload_view(h, d[1], lv.d32.y)) || (rc = upload_view(h, d[2], lv.d32.z)))
      return bail(rc);
    lv.nodes = (long)d[0].N * d[1].N * d[2].N;
    if (l == L)
      for (int a = 0; a < 3; ++a) h->coords[a] = d[a].coords;
    char* b;
    for (void** v : {&lv.u, &lv.f, &lv.r}) {
      if ((rc = alloc3(h, &b, lv.nodes * tsz))) return bail(rc);
      CK3(cudaMemset(b, 0, lv.nodes * tsz));
      *v = b;
    }
    if (l > 0) {
      if ((rc = alloc3(h, &b, (size_t)ne * lv.m * lv.m * lv.m * tsz))) return bail(rc);
      lv.E = b;
      const int nc = lv.p / 2 + 1;
      if ((rc = alloc3(h, &b, (size_t)ne * nc * nc * nc * tsz))) return bail(rc);
      lv.Ec = b;
      std::vector<double> J;
      interp_matrix(lv.p, lv.p / 2, J);
      if ((rc = upload3(h, &lv.J64, J)) || (rc = upload3(h, &lv.J32, J))) return bail(rc);
    }
  }
  // coarse fast diagonalisation
  {
    long nu = 1;
    for (int a = 0; a < 3; ++a) {
      Coarse1D cd;
      const std::string err = build_coarse(ms[a], cd);
      if (!err.empty()) {
        sem3_destroy(h);
        return fail3(SEM_BAD_ARG, err);
      }
      h->c64.nu[a] = h->c32.nu[a] = cd.nu;
      h->c64.first[a] = h->c32.first[a] = cd.first;
      h->c64.N[a] = h->c32.N[a] = ms[a].nodes(1);
      double *S, *l64;
      float *S32, *l32;
      if ((rc = upload3(h, &S, cd.S)) || (rc = upload3(h, &l64, cd.lam)) || (rc = upload3(h, &S32, cd.S)) ||
          (rc = upload3(h, &l32, cd.lam)))
        return bail(rc);
      h->c64.S[a] = S;
      h->c64.lam[a] = l64;
      h->c32.S[a] = S32;
      h->c32.lam[a] = l32;
      nu *= cd.nu;
    }
    h->c64.singular = h->c32.singular = per ? 1 : 0;
    char* b;
    if ((rc = alloc3(h, &b, nu * tsz))) return bail(rc);
    h->cw1 = b;
    if ((rc = alloc3(h, &b, nu * tsz))) return bail(rc);
    h->cw2 = b;
  }
  h->n = h->lev[L].nodes;
  h->n_unknowns = per ? (long)c.nx * c.p * c.ny * c.p * c.nz * c.p
                      : (long)(c.nx * c.p - 1) * (c.ny * c.p - 1) * (c.nz * c.p - 1);
  for (double** v : {&h->r, &h->p, &h->q, &h->z, &h->r_old}) {
    if ((rc = alloc3(h, v, h->n))) return bail(rc);
    CK3(cudaMemset(*v, 0, h->n * sizeof(double)));
  }
  if ((rc = alloc3(h, &h->part, kDot3Parts))) return bail(rc);
  if (per) {
    if ((rc = alloc3(h, &h->ones, h->n))) return bail(rc);
    std::vector<double> one(h->n, 1.0);
    CK3(cudaMemcpy(h->ones, one.data(), h->n * sizeof(double), cudaMemcpyHostToDevice));
  }
  CK3(cudaDeviceSynchronize());
  *out = h;
  return SEM_OK;
}

int sem3_sizes(const sem3_handle* h, int64_t* n_unknowns, int64_t* nx, int64_t* ny, int64_t* nz) {
  if (!h) return fail3(SEM_BAD_ARG, "null handle");
  if (n_unknowns) *n_unknowns = h->n_unknowns;
  if (nx) *nx = (int64_t)h->coords[0].size();
  if (ny) *ny = (int64_t)h->coords[1].size();
  if (nz) *nz = (int64_t)h->coords[2].size();
  return SEM_OK;
}

int sem3_coords(const sem3_handle* h, double* x, double* y, double* z) {
  if (!h) return fail3(SEM_BAD_ARG, "null handle");
  double* dst[3] = {x, y, z};
  for (int a = 0; a < 3; ++a)
    if (dst[a]) std::memcpy(dst[a], h->coords[a].data(), h->coords[a].size() * sizeof(double));
  return SEM_OK;
}

int sem3_mass(sem3_handle* h, const double* f, double* b, void* stream) {
  int rc = check3(h);
  if (rc) return rc;
  if (!f || !b) return fail3(SEM_BAD_ARG, "null vector");
  cudaStream_t s = st3(stream);
  CK3((launch3_mass<double>(h->lev[h->L].d64, f, b, s)));
  if (h->ones) {  // periodic: project onto the range of A (zero mean)
    double sum = 0.0;
    if ((rc = dot3(h, b, h->ones, &sum, s))) return rc;
    CK3(launch3_axpby(h->n, -sum / (double)h->n, h->ones, 1.0, b, s));
  }
  return SEM_OK;
}

int sem3_apply(sem3_handle* h, const double* u, double* Au, void* stream) {
  int rc = check3(h);
  if (rc) return rc;
  if (!u || !Au) return fail3(SEM_BAD_ARG, "null vector");
  CK3((launch3_apply<double, double>(h->lev[h->L].d64, u, nullptr, Au, st3(stream))));
  return SEM_OK;
}

int sem3_smooth(sem3_handle* h, double* u, const double* f, int32_t n_it, void* stream) {
  int rc = check3(h);
  if (rc) return rc;
  if (!u || !f || n_it < 0) return fail3(SEM_BAD_ARG, "invalid argument");
  cudaStream_t s = st3(stream);
  const Level3& top = h->lev[h->L];
  for (int k = 0; k < n_it; ++k) {
    CK3((launch3_apply<double, double>(top.d64, u, f, h->r, s)));
    if (h->mixed) {
      float* r32 = static_cast<float*>(top.r);
      CK3((launch3_convert<double, float>(h->n, h->r, r32, s)));
      CK3((launch3_sweep<float, double>(top.d32, r32, static_cast<float*>(top.E), u, true, s)));
    } else {
      CK3((launch3_sweep<double, double>(top.d64, h->r, static_cast<double*>(top.E), u, true, s)));
    }
  }
  return SEM_OK;
}

int sem3_vcycle(sem3_handle* h, double* u, const double* f, void* stream) {
  int rc = check3(h);
  if (rc) return rc;
  if (!u || !f) return fail3(SEM_BAD_ARG, "null vector");
  cudaStream_t s = st3(stream);
  // MultigridCycle(u, f) = u + MultigridCycle(0, f - A u): the cycle is affine
  CK3((launch3_apply<double, double>(h->lev[h->L].d64, u, f, h->r, s)));
  if ((rc = precond3(h, h->r, h->z, s))) return rc;
  CK3(launch3_axpby(h->n, 1.0, h->z, 1.0, u, s));
  return SEM_OK;
}

int sem3_pcg_solve(sem3_handle* h, double* u, const double* f, sem_result* res, double* history, int32_t hlen,
                   void* stream) {
  int rc = check3(h);
  if (rc) return rc;
  if (!u || !f || !res) return fail3(SEM_BAD_ARG, "null argument");
  cudaStream_t s = st3(stream);
  const long n = h->n;
  const Dir3<double>& d = h->lev[h->L].d64;
  std::memset(res, 0, sizeof(*res));
  auto put = [&](int i, double v) {
    if (history && i < hlen) history[i] = v;
  };
  double rr;
  CK3((launch3_apply<double, double>(d, u, f, h->r, s)));
  if ((rc = dot3(h, h->r, h->r, &rr, s))) return rc;
  res->res0 = res->res = std::sqrt(rr);
  put(0, res->res0);
  if (res->res0 == 0.0) {
    res->status = SEM_OK;
    return SEM_OK;
  }
  const double rmax = h->cfg.tol * res->res0;
  CK3(cudaMemsetAsync(h->r_old, 0, n * sizeof(double), s));
  if ((rc = precond3(h, h->r, h->p, s))) return rc;
  double delta;
  if ((rc = dot3(h, h->p, h->r, &delta, s))) return rc;
  int status = SEM_NOT_CONVERGED;
  int it = 0;
  for (int i = 1; i <= h->cfg.i_max; ++i) {
    it = i;
    CK3((launch3_apply<double, double>(d, h->p, nullptr, h->q, s)));
    double pq;
    if ((rc = dot3(h, h->p, h->q, &pq, s))) return rc;
    if (!(pq > 0.0) || !std::isfinite(delta)) {
      status = SEM_BREAKDOWN;
      break;
    }
    const double alpha = delta / pq;
    CK3(launch3_axpby(n, alpha, h->p, 1.0, u, s));
    CK3(cudaMemcpyAsync(h->r_old, h->r, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    CK3(launch3_axpby(n, -alpha, h->q, 1.0, h->r, s));
    if ((rc = dot3(h, h->r, h->r, &rr, s))) return rc;
    res->res = std::sqrt(rr);
    put(i, res->res);
    if (!std::isfinite(res->res)) {
      status = SEM_BREAKDOWN;
      break;
    }
    if (res->res <= rmax) {
      status = SEM_OK;
      break;
    }
    if ((rc = precond3(h, h->r, h->z, s))) return rc;
    // beta = z^T (r - r_old) / delta (Polak-Ribiere), r_old = 0 before the first update
    double zr, zro;
    if ((rc = dot3(h, h->z, h->r, &zr, s)) || (rc = dot3(h, h->z, h->r_old, &zro, s))) return rc;
    const double beta = (i == 1 ? zr : zr - zro) / delta;
    CK3(launch3_axpby(n, 1.0, h->z, beta, h->p, s));
    delta = zr;
  }
  res->iterations = it;
  res->status = status;
  res->rbar = it > 0 && res->res > 0 ? std::log10(res->res0 / res->res) / it : 0.0;
  return status;
}

}  // extern "C"

"""CPU-side checks of the C-ABI library: it loads, exports every symbol that
include/sem_schwarz.h declares, validates configurations, and its host FP64
set-up tables (GLL coordinates, fast-diagonalisation factors, weights) agree
with the oracle.  No GPU is needed; no kernel is launched."""
import os
import re

import numpy as np
import pytest

from oracle import sem_oracle as O

P = pytest.importorskip("paper_1512_02390_gb300")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            names |= set(re.findall(r"^\s*(?:int|int64_t|void|const char\*)\s+(sem_\w+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    try:
        return P.load_library()
    except RuntimeError as e:
        pytest.skip(str(e))


def test_library_exports_every_declared_symbol(lib):
    decl = _declared_symbols()
    assert len(decl) >= 13
    for name in decl:
        assert hasattr(lib, name), name
    assert decl <= set(P.EXPORTS)


def test_bad_configs_are_rejected_on_the_host(lib):
    for kw in [dict(p=6), dict(p=64), dict(nx=1), dict(weight=2), dict(precision=9), dict(tol=-1.0)]:
        cfg = P.sem_default_config()
        for k, v in kw.items():
            setattr(cfg, k, v)
        with pytest.raises(P.SemError) as ei:
            P.sem_inspect_level(cfg, 1)
        assert ei.value.status == P.SEM_BAD_ARG


def _oracle_level(periodic, nx, p, n_o, weight, edges=None, length=1.0):
    mx = O.Mesh1D.uniform(nx, length, periodic) if edges is None else O.Mesh1D(np.asarray(edges), periodic)
    return O.Level(mx, O.Mesh1D.uniform(3, 1.0, periodic), p, n_o, weight=weight)


@pytest.mark.parametrize("periodic,nx,p,overlap,weight,edges", [
    (False, 4, 4, 1, 5, None), (True, 8, 16, 2, 5, None), (False, 5, 8, 3, "a", None),
    (False, 4, 32, 4, 7, None), (True, 6, 4, 1, "t", None), (False, 4, 8, 2, 3, [0.0, 0.1, 0.4, 0.45, 1.0]),
    (False, 3, 2, 1, 1, None)])
def test_host_tables_match_oracle(lib, periodic, nx, p, overlap, weight, edges):
    cfg = P.make_config(nx=nx, ny=3, p=p, periodic=periodic, overlap=overlap, weight=weight, x_edges=edges)
    L = int(np.log2(p))
    t = P.sem_inspect_level(cfg, L)
    lev = _oracle_level(periodic, nx, p, t["n_o"], weight, edges)
    assert t["p"] == p and t["m"] == p + 1 + 2 * t["n_o"]
    np.testing.assert_allclose(t["coords"], lev.mx.coords(p), atol=1e-14)
    m, no = t["m"], t["n_o"]
    for e in range(nx):
        s = lev.sub_x[e]
        slots = s.k + no
        tid = t["tab"][e]
        # weights over the valid window slots, zero elsewhere
        w = np.zeros(m)
        w[slots] = s.w
        np.testing.assert_allclose(t["w"][tid], w, atol=1e-14)
        # eigen-decomposition of the restricted pair: same spectrum, and the
        # library's vectors diagonalise the oracle's restricted (L~, M~)
        mv = len(slots)
        np.testing.assert_allclose(t["lam"][tid][:mv], s.lam, rtol=1e-11, atol=1e-11 * s.lam.max())
        Sv = t["S"][tid][slots][:, :mv]
        Mt = np.diag(lev.Mx_glob[s.g])
        Lt = lev.Lx_glob[np.ix_(s.g, s.g)]
        np.testing.assert_allclose(Sv.T @ Mt @ Sv, np.eye(mv), atol=1e-11)
        np.testing.assert_allclose(Sv.T @ Lt @ Sv, np.diag(s.lam), atol=1e-10 * s.lam.max())
        # padding: zero rows outside the window, unit eigenvalue slots
        pad = np.setdiff1d(np.arange(m), slots)
        assert np.all(t["S"][tid][pad] == 0) and np.all(t["lam"][tid][mv:] == 1.0)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 7, 8, 16, 32, 64])
def test_gll_tables_equal_the_oracle_bitwise(lib, p):
    """The library's 1D set (double-double arithmetic, rounded once) and the
    oracle's (50-digit decimal, rounded once) are both the correctly rounded
    values, so they agree bit for bit although no code is shared."""
    xi, w, D, L = P.sem_gll_tables(p)
    oxi, ow = O.gll(p)
    _, oL = O.element_matrices(p, 2.0)
    for a, b in ((xi, oxi), (w, ow), (D, O.gll_diff(p)), (L, oL)):
        assert np.array_equal(a, b)


def test_gll_tables_reject_bad_order(lib):
    for p in (0, 65):
        with pytest.raises(P.SemError):
            P.sem_gll_tables(p)


# ---- the integer binary64 -> binary32 rounding of the MGCG update -------------

_CONV_SRC = r'''
#include "f32_round.h"
extern "C" void conv(const double* x, float* y, long n) {
  for (long i = 0; i < n; ++i) y[i] = sem::f32_from_f64_rn(x[i]);
}
'''


def test_f32_rounding_matches_ieee_round_to_nearest_even(tmp_path):
    """The FP32 copy of r is rounded by integer operations on the bit fields;
    it must equal IEEE round-to-nearest-even (numpy's float64 -> float32)
    bit for bit: random values over every binary32 binade and beyond, exact
    ties on both parities, the largest binade's carry to infinity, the
    subnormal boundary, zeros, infinities and NaN."""
    import ctypes
    import shutil
    import subprocess
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    src = tmp_path / "conv.cpp"
    src.write_text(_CONV_SRC)
    so = tmp_path / "conv.so"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_1512_02390_gb300", "csrc")
    subprocess.run(["g++", "-O2", "-shared", "-fPIC", "-I", inc, str(src), "-o", str(so)], check=True)
    f = ctypes.CDLL(str(so)).conv
    rng = np.random.default_rng(5)
    n = 400000
    x = np.ldexp(rng.uniform(0.5, 1.0, n), rng.integers(-160, 140, n)) * rng.choice([-1.0, 1.0], n)
    # exact ties: a binary32 value plus half its ulp (even and odd last bits)
    base = np.ldexp(rng.uniform(1.0, 2.0, 2000).astype(np.float32).astype(np.float64), rng.integers(-120, 120, 2000))
    ulp = np.spacing(base.astype(np.float32)).astype(np.float64)
    ties = np.concatenate([base + 0.5 * ulp, base - 0.5 * ulp * (base.astype(np.float32) != base)])
    fmax = float(np.finfo(np.float32).max)
    edge = np.array([0.0, -0.0, np.inf, -np.inf, fmax, -fmax, fmax * (1 + 2.0**-25), fmax * (1 + 2.0**-24),
                     fmax + 2.0**103, np.nextafter(fmax + 2.0**103, 0), 2.0**128, 2.0**-126,
                     np.nextafter(2.0**-126, 0), 2.0**-127, 2.0**-149, 2.0**-150, 3 * 2.0**-151, 1e-300,
                     1e300, 1.0, -1.0, 1 + 2.0**-24, 1 + 3 * 2.0**-24, 1 + 2.0**-24 + 2.0**-52])
    x = np.ascontiguousarray(np.concatenate([x, ties, edge]), dtype=np.float64)
    y = np.empty(x.size, dtype=np.float32)
    f(x.ctypes.data_as(ctypes.c_void_p), y.ctypes.data_as(ctypes.c_void_p), ctypes.c_long(x.size))
    with np.errstate(over="ignore"):
        want = x.astype(np.float32)
    assert np.array_equal(y.view(np.uint32), want.view(np.uint32))
    z = np.array([np.nan], dtype=np.float64)
    f(z.ctypes.data_as(ctypes.c_void_p), y.ctypes.data_as(ctypes.c_void_p), ctypes.c_long(1))
    assert np.isnan(y[0])


_TF32_SRC = r'''
#include "f32_round.h"
extern "C" void tf32(const unsigned* x, unsigned* y, long n) {
  for (long i = 0; i < n; ++i) y[i] = sem::tf32_bits_rna(x[i]);
}
'''


def test_tf32_rounding_is_round_to_nearest_ties_away(tmp_path):
    """The tensor-core operands are rounded to TF32 by integer operations on
    the binary32 bits; the result must be the nearer of the two neighbouring
    TF32 values (10 fraction bits), ties away from zero, computed here by
    exact float64 arithmetic: random values over the normal binades, exact
    ties, values just below and above a tie, a carry into the next binade,
    and zeros."""
    import ctypes
    import shutil
    import subprocess
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    src = tmp_path / "tf32.cpp"
    src.write_text(_TF32_SRC)
    so = tmp_path / "tf32.so"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_1512_02390_gb300", "csrc")
    subprocess.run(["g++", "-O2", "-shared", "-fPIC", "-I", inc, str(src), "-o", str(so)], check=True)
    f = ctypes.CDLL(str(so)).tf32
    rng = np.random.default_rng(7)
    n = 200000
    x = (np.ldexp(rng.uniform(1.0, 2.0, n), rng.integers(-120, 120, n)) * rng.choice([-1.0, 1.0], n)).astype(np.float32)
    # exact ties and their neighbours: a TF32 value plus half its unit, plus / minus one binary32 ulp
    t = np.ldexp(rng.integers(1024, 2048, 3000).astype(np.float64) / 1024.0, rng.integers(-100, 100, 3000))
    half = np.ldexp(1.0, np.frexp(t)[1] - 12)   # half a TF32 unit of t
    ties = (t + half).astype(np.float32)
    near = np.concatenate([ties, np.nextafter(ties, np.float32(0)), np.nextafter(ties, np.float32(np.inf)), -ties])
    edge = np.array([0.0, -0.0, 1.0, -1.0, 2.0 - 2.0**-11, 2.0 - 2.0**-23, 1.0 + 2.0**-11, 1.0 + 2.0**-12],
                    dtype=np.float32)
    x = np.ascontiguousarray(np.concatenate([x, near, edge]).astype(np.float32))
    y = np.empty(x.size, dtype=np.uint32)
    f(x.ctypes.data_as(ctypes.c_void_p), y.ctypes.data_as(ctypes.c_void_p), ctypes.c_long(x.size))
    got = y.view(np.float32).astype(np.float64)
    v = x.astype(np.float64)
    mag = np.abs(v)
    with np.errstate(divide="ignore"):
        e = np.where(mag > 0, np.frexp(mag)[1] - 1, 0)   # v = m 2^e, 1 <= m < 2
    unit = np.ldexp(1.0, e - 10)                          # TF32 unit in the binade of v
    lo = np.floor(mag / unit) * unit
    hi = lo + unit
    want = np.where(mag - lo < hi - mag, lo, hi) * np.sign(v)
    want = np.where(mag - lo == hi - mag, hi * np.sign(v), want)   # ties away from zero
    want = np.where(mag == 0, v, want)
    assert np.array_equal(got, want)
    assert np.all((y & 0x1FFF) == 0)


# ---- the exact fixed-point conversions of the integer FP64 operator ----------

_FX_SRC = r'''
#include "fx_exact.h"
extern "C" void to_f64(const long long* c, const int* K, double* y, long n) {
  for (long i = 0; i < n; ++i) y[i] = sem::fx_to_f64(c[4 * i], c[4 * i + 1], c[4 * i + 2], c[4 * i + 3], K[i]);
}
extern "C" void of(const double* x, const int* emax, long long* X, long n) {
  for (long i = 0; i < n; ++i) X[i] = sem::fx_of(x[i], emax[i]);
}
extern "C" void limbs(const long long* v, int* lo, int* hi, long n) {
  for (long i = 0; i < n; ++i) sem::fx_limbs(v[i], lo[i], hi[i]);
}
'''


def _fx_lib(tmp_path):
    import ctypes
    import shutil
    import subprocess
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    src = tmp_path / "fx.cpp"
    src.write_text(_FX_SRC)
    so = tmp_path / "fx.so"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                       "paper_1512_02390_gb300", "csrc")
    subprocess.run(["g++", "-O2", "-shared", "-fPIC", "-I", inc, str(src), "-o", str(so)], check=True)
    return ctypes.CDLL(str(so))


def test_fixed_point_sum_rounds_like_exact_rational_arithmetic(tmp_path):
    """The integer FP64 operator turns four int64 accumulators (weights 2^0,
    2^25, 2^50, 2^75, not carry-normalised, |c| < 2^62) times 2^-K into a
    double.  Python's exact integers and its correctly rounded int -> float
    division give the reference: every normal result must match bit for bit.
    Cases: magnitudes of 1 to 136 bits of both signs, exact ties at the
    rounding bit on both parities with their neighbours, carries spread over
    the limbs in random ways, zero."""
    import ctypes
    from fractions import Fraction
    lib = _fx_lib(tmp_path)
    rng = np.random.default_rng(11)
    vals = []
    for nb in range(1, 137):
        for _ in range(12):
            v = int(rng.integers(1, 2**62)) << max(0, nb - 62)
            v = (v | 1) & ((1 << nb) - 1) | (1 << (nb - 1))
            vals.append(v if rng.random() < 0.5 else -v)
    for _ in range(600):  # ties at the 53-bit rounding position and their neighbours
        g = int(rng.integers(0, 80))
        m = int(rng.integers(2**52, 2**53))
        t = (2 * m + 1) << g
        for v in (t, t - 1, t + 1):
            vals.append(v if rng.random() < 0.5 else -v)
    vals.append(0)
    cs, Ks, want = [], [], []
    B = 1 << 25
    for v in vals:
        c = [0, 0, 0, 0]
        r = v
        for i in range(3):  # canonical limbs, then move random carries between them
            c[i] = r % B
            r //= B
        c[3] = r
        for i in range(3):
            a = int(rng.integers(-2**30, 2**30))
            c[i] += a * B
            c[i + 1] -= a
        assert all(abs(x) < 2**62 for x in c)
        assert c[0] + c[1] * B + c[2] * B**2 + c[3] * B**3 == v
        top = abs(v).bit_length()
        K = int(top + rng.integers(-1000, 1000)) if v else 5
        w = float(Fraction(v, 1 << K)) if K >= 0 else float(v * (1 << -K))
        if v and not (2.0**-1022 <= abs(w) < 2.0**1023):
            continue
        cs.append(c)
        Ks.append(K)
        want.append(w)
    c = np.ascontiguousarray(np.array(cs, dtype=np.int64))
    K = np.ascontiguousarray(np.array(Ks, dtype=np.int32))
    y = np.empty(len(Ks))
    lib.to_f64(c.ctypes.data_as(ctypes.c_void_p), K.ctypes.data_as(ctypes.c_void_p),
               y.ctypes.data_as(ctypes.c_void_p), ctypes.c_long(len(Ks)))
    assert np.array_equal(y.view(np.uint64), np.array(want).view(np.uint64))


def test_fixed_point_operand_and_limbs_are_exact(tmp_path):
    """A staged double becomes X = x 2^(1075 - emax) rounded to the nearest
    integer (ties away from zero), |X| < 2^53, and X +- X' splits exactly into
    lo + hi 2^25 with lo in [0, 2^25)."""
    import ctypes
    from fractions import Fraction
    lib = _fx_lib(tmp_path)
    rng = np.random.default_rng(12)
    n = 20000
    x = np.ldexp(rng.uniform(0.5, 1.0, n), rng.integers(-1000, 1000, n)) * rng.choice([-1.0, 1.0], n)
    ex = (x.view(np.uint64) >> np.uint64(52)) & np.uint64(0x7ff)
    emax = (ex.astype(np.int64) + rng.integers(0, 60, n)).astype(np.int32)
    x = np.concatenate([x, [0.0, -0.0, 2.0**-1074, 1.5, -1.5]])
    emax = np.concatenate([emax, np.array([1023, 1023, 1023, 1023 + 53, 1023 + 53], dtype=np.int32)])
    X = np.empty(x.size, dtype=np.int64)
    lib.of(np.ascontiguousarray(x).ctypes.data_as(ctypes.c_void_p), np.ascontiguousarray(emax).ctypes.data_as(ctypes.c_void_p),
           X.ctypes.data_as(ctypes.c_void_p), ctypes.c_long(x.size))
    for xi, ei, Xi in zip(x, emax, X):
        b = int(np.float64(xi).view(np.uint64))
        if (b >> 52) & 0x7ff == 0:
            assert Xi == 0
            continue
        q = Fraction(float(xi)) * Fraction(2) ** (1075 - int(ei))
        r = int(abs(q) + Fraction(1, 2))  # nearest, ties away from zero
        assert Xi == (r if q >= 0 else -r) and abs(int(Xi)) < 2**53
    v = np.concatenate([rng.integers(-2**54 + 1, 2**54, 5000), [0, -1, 1, 2**25, -2**25, 2**54 - 1, -2**54 + 1]])
    v = np.ascontiguousarray(v.astype(np.int64))
    lo = np.empty(v.size, dtype=np.int32)
    hi = np.empty(v.size, dtype=np.int32)
    lib.limbs(v.ctypes.data_as(ctypes.c_void_p), lo.ctypes.data_as(ctypes.c_void_p), hi.ctypes.data_as(ctypes.c_void_p),
              ctypes.c_long(v.size))
    assert np.all((lo >= 0) & (lo < 2**25))
    assert np.array_equal(lo.astype(np.int64) + hi.astype(np.int64) * 2**25, v)


# ---- the fixed-point element tables of the integer FP64 operator ----------

_FXTAB_SRC = r'''
#include <cstring>
#include "setup.h"
extern "C" int fx_tab(int n, const double* edges, int periodic, int p, int n_o, int* tab, int tab_cap, int* t,
                      int* slot, int* ntab, double* Le) {
  sem::Mesh1D m;
  m.n = n;
  m.periodic = periodic != 0;
  m.edges.assign(edges, edges + n + 1);
  sem::Dir1D d;
  if (!sem::build_dir(m, p, n_o, 5, d).empty()) return -1;
  std::vector<int> tb, tt, sl;
  if (!sem::fx_tables(d, tb, tt, sl)) return -2;
  if ((int)tb.size() > tab_cap) return -3;
  std::memcpy(tab, tb.data(), tb.size() * sizeof(int));
  std::memcpy(t, tt.data(), tt.size() * sizeof(int));
  std::memcpy(slot, sl.data(), sl.size() * sizeof(int));
  *ntab = (int)tt.size();
  std::memcpy(Le, d.Le.data(), d.Le.size() * sizeof(double));
  return 0;
}
'''


@pytest.mark.parametrize("edges,p,periodic", [
    ([0.0, 0.25, 0.5, 0.625, 0.75, 1.0], 8, False),      # two element widths, interleaved
    ([i / 6 for i in range(7)], 16, False),                # uniform (computed edges: widths may differ in the last bit)
    ([0.0, 0.5, 0.75, 0.875, 0.9375, 1.0], 32, False),     # five widths
    ([0.0, 0.25, 0.375, 0.5, 0.75, 1.0], 4, True),         # periodic
])
def test_fixed_point_tables_are_exact_and_shared(tmp_path, edges, p, periodic):
    """The operator's element tables (setup.cpp fx_tables): every element
    matrix L becomes L_int = L 2^t, which must be an exact integer with
    2^72 <= max |L_int| < 2^73; the even-odd entries E[a][k] = L_int[a][k] +
    L_int[a][p-k] (E[a][p/2] = 2 L_int[a][p/2]) and O[a][k] = L_int[a][k] -
    L_int[a][p-k] are stored as three 25-bit limbs l2 2^50 + l1 2^25 + l0.
    Elements with bitwise equal matrices share one table, others do not, and
    the last table (that of the missing neighbour) is zero.  Checked against
    Python's exact rational arithmetic on the library's own element matrices."""
    import ctypes
    import shutil
    import subprocess
    from fractions import Fraction
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    csrc = os.path.join(root, "paper_1512_02390_gb300", "csrc")
    src = tmp_path / "fxtab.cpp"
    src.write_text(_FXTAB_SRC)
    so = tmp_path / "fxtab.so"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-I", csrc, "-I",
                    os.path.join(root, "include"), os.path.join(csrc, "setup.cpp"), str(src), "-o", str(so)],
                   check=True)
    lib = ctypes.CDLL(str(so))
    n, H, np1 = len(edges) - 1, p // 2, p + 1
    NE, NO = (H + 1) ** 2, H * H
    EO = NE + NO
    cap = (n + 1) * EO * 4
    tab = np.zeros(cap, dtype=np.int32)
    t = np.zeros(n + 1, dtype=np.int32)
    slot = np.zeros(n + 1, dtype=np.int32)
    ntab = ctypes.c_int(0)
    Le = np.zeros(n * np1 * np1)
    e = np.ascontiguousarray(np.array(edges, dtype=np.float64))
    vp = ctypes.c_void_p
    rc = lib.fx_tab(ctypes.c_int(n), e.ctypes.data_as(vp), ctypes.c_int(int(periodic)), ctypes.c_int(p),
                    ctypes.c_int(1), tab.ctypes.data_as(vp), ctypes.c_int(cap), t.ctypes.data_as(vp),
                    slot.ctypes.data_as(vp), ctypes.byref(ntab), Le.ctypes.data_as(vp))
    assert rc == 0
    k = ntab.value
    tab = tab[:k * EO * 4].reshape(k, EO, 4).astype(np.int64)
    # sharing: equal matrices <=> equal table; the zero table last
    rows = [Le[i * np1 * np1:(i + 1) * np1 * np1].tobytes() for i in range(n)]
    assert len(set(rows)) == k - 1
    for i in range(n):
        for j in range(n):
            assert (slot[i] == slot[j]) == (rows[i] == rows[j])
    assert slot[n] == k - 1 and t[k - 1] == 0 and not tab[k - 1].any()
    assert sorted(set(slot[:n].tolist())) == list(range(k - 1))
    # exact fixed point, even-odd folding and limbs
    assert np.all((tab[..., 0] >= 0) & (tab[..., 0] < 2**25) & (tab[..., 1] >= 0) & (tab[..., 1] < 2**25))
    assert not tab[..., 3].any()
    val = [[int(x[2]) * 2**50 + int(x[1]) * 2**25 + int(x[0]) for x in tab[s]] for s in range(k)]
    for i in range(n):
        s, te = slot[i], int(t[slot[i]])
        L = Le[i * np1 * np1:(i + 1) * np1 * np1].reshape(np1, np1)
        Li = [[Fraction(float(L[a, b])) * Fraction(2) ** te for b in range(np1)] for a in range(np1)]
        assert all(x.denominator == 1 for row in Li for x in row)
        Li = [[int(x) for x in row] for row in Li]
        big = max(abs(x) for row in Li for x in row)
        assert 2**72 <= big < 2**73
        for a in range(H + 1):
            for kk in range(H + 1):
                want = 2 * Li[a][H] if kk == H else Li[a][kk] + Li[a][p - kk]
                assert val[s][a * (H + 1) + kk] == want
        for a in range(H):
            for kk in range(H):
                assert val[s][NE + a * H + kk] == Li[a][kk] - Li[a][p - kk]


def test_noalloc_wrapper_rejects_vectors_of_the_wrong_size():
    """The Python wrapper of the allocation-free correction checks r and u
    against the node grid the tables describe (n p + 1 nodes per Dirichlet
    direction, n p periodic) before any call into the library, which cannot
    check pointer extents itself."""
    torch = pytest.importorskip("torch")
    P = pytest.importorskip("paper_1512_02390_gb300")
    tx = P.sem_sweep_tables(n=4, p=8, n_o=1, periodic=0)
    ty = P.sem_sweep_tables(n=3, p=8, n_o=1, periodic=0)
    ok = torch.zeros((3 * 8 + 1) * (4 * 8 + 1), dtype=torch.float64)
    short = torch.zeros(ok.numel() - 1, dtype=torch.float64)
    for r, u in ((short, ok), (ok, short), (ok[: (4 * 8 + 1) ** 2 - 8], ok)):
        with pytest.raises(ValueError):
            P.sem_schwarz_correction_noalloc(tx, ty, r, u)
    px = P.sem_sweep_tables(n=4, p=8, n_o=1, periodic=1)
    py = P.sem_sweep_tables(n=3, p=8, n_o=1, periodic=1)
    with pytest.raises(ValueError):  # a periodic grid has 24 x 32 nodes
        P.sem_schwarz_correction_noalloc(px, py, ok, ok)

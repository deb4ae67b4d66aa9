"""Plain FP64 CPU oracle of the three-dimensional extension of the hybrid
Schwarz/multigrid spectral-element solver (the paper's concluding section
names the extension to three space dimensions as future work).

TEST INFRASTRUCTURE ONLY.  Like ``sem_oracle`` (whose one-dimensional
building blocks it reuses: GLL set, element matrices, assembly, the
extended-element windows of Sec. 3.1 with their restricted 1D eigenpairs and
weights), it may be imported only by the test-suite, the smoke check and the
CPU legs of ``bench.py``; the product library never imports it.

What carries over from the 2D method, one dimension up:
  * Eq. (system matrix) in 3D, A = M_z (x) M_y (x) L_x + M_z (x) L_y (x) M_x
    + L_z (x) M_y (x) M_x, applied element by element with explicit gather
    and scatter-add (diagonal GLL mass, reading R1).
  * Sec. 3.1 subdomains: the extended element is the tensor product of the
    1D windows (n_o node layers adopted from each neighbour, outer layer
    excluded), so A_ss keeps the tensor form and its inverse is the
    fast-diagonalisation product with three contractions on each side,
        A_ss^{-1} = (S_z (x) S_y (x) S_x) (I (x) I (x) Lam_x + I (x) Lam_y (x) I
                    + Lam_z (x) I (x) I)^{-1} (S_z^T (x) S_y^T (x) S_x^T),
    and the weights of Eq. (weight function) are W = W_z (x) W_y (x) W_x
    (for w_a the counting matrix is the tensor product of the 1D counts).
  * Alg. 2 (weighted additive Schwarz), Alg. 3 (V-cycle with the embedded
    interpolation I_l = P_z (x) P_y (x) P_x and its transpose, coarse
    pseudo-inverse A_0^+ by a dense Cholesky), Alg. 4 (MGCG, beta line read
    as z^T (r - r_old) / delta, reading R6).
Each direction may be periodic or have Dirichlet walls.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla

from .sem_oracle import Level as _Level2
from .sem_oracle import Mesh1D, overlap_rule, prolongation_1d


class Dir:
    """One direction at order p: element matrices, assembled 1D matrices,
    unknown mask and the 1D subdomain factors (windows, eigenpairs, weights)
    of every element, taken from the 2D oracle's per-direction set-up."""

    def __init__(self, mesh: Mesh1D, p: int, n_o: int, weight=5):
        lev = _Level2(mesh, mesh, p, n_o, weight=weight)
        self.mesh, self.p, self.n_o = mesh, p, n_o
        self.M, self.L = lev.Mx, lev.Lx          # per element: mass diagonal, stiffness
        self.Mg = lev.Mx_glob                     # assembled mass diagonal
        self.g = lev.gx                           # gidx[e, k]
        self.N = lev.NX
        self.unknown = mesh.unknown(p)
        self.subs = lev.sub_x                     # Sub1D per element: g, k, S, lam, w


class Level3:
    """Operator and Schwarz data at order p on an nx x ny x nz Cartesian mesh.
    Fields are arrays of shape (NZ, NY, NX), x fastest."""

    def __init__(self, mx: Mesh1D, my: Mesh1D, mz: Mesh1D, p: int, n_o: int, weight=5):
        self.p, self.n_o = p, n_o
        self.dx, self.dy, self.dz = Dir(mx, p, n_o, weight), Dir(my, p, n_o, weight), Dir(mz, p, n_o, weight)
        self.NX, self.NY, self.NZ = self.dx.N, self.dy.N, self.dz.N
        self.shape = (self.NZ, self.NY, self.NX)
        self.unknown = (self.dz.unknown[:, None, None] & self.dy.unknown[None, :, None]
                        & self.dx.unknown[None, None, :])
        self.periodic = mx.periodic and my.periodic and mz.periodic

    def apply(self, u: np.ndarray) -> np.ndarray:
        """A u, Eq. (system matrix) in 3D, element by element."""
        dx, dy, dz = self.dx, self.dy, self.dz
        u = np.where(self.unknown, u, 0.0)
        GZ = dz.g[:, None, None, :, None, None]
        GY = dy.g[None, :, None, None, :, None]
        GX = dx.g[None, None, :, None, None, :]
        U = u[GZ, GY, GX]  # (ez, ey, ex, k, j, i): gather of the element coefficients
        mz = dz.M[:, None, None, :, None, None]
        my = dy.M[None, :, None, None, :, None]
        mx = dx.M[None, None, :, None, None, :]
        V = (mz * my * np.einsum("xab,zyxkjb->zyxkja", dx.L, U)
             + mz * mx * np.einsum("yab,zyxkbi->zyxkai", dy.L, U)
             + my * mx * np.einsum("zab,zyxbji->zyxaji", dz.L, U))
        flat = np.broadcast_to((GZ * self.NY + GY) * self.NX + GX, V.shape)
        out = np.bincount(flat.ravel(), weights=V.ravel(), minlength=self.NZ * self.NY * self.NX)
        return np.where(self.unknown, out.reshape(self.shape), 0.0)

    def mass(self, f_nodal: np.ndarray) -> np.ndarray:
        """b = (M_z (x) M_y (x) M_x) f; projected to zero mean when A is singular."""
        b = self.dz.Mg[:, None, None] * self.dy.Mg[None, :, None] * self.dx.Mg[None, None, :] * f_nodal
        b = np.where(self.unknown, b, 0.0)
        if self.periodic:
            b = b - b.mean()
        return b

    def local_solve(self, ex: int, ey: int, ez: int, rs: np.ndarray) -> np.ndarray:
        """Delta u_s = A_ss^{-1} r_s by fast diagonalisation: three contractions
        with S^T, the division by lam_z + lam_y + lam_x, three with S."""
        sx, sy, sz = self.dx.subs[ex], self.dy.subs[ey], self.dz.subs[ez]
        X = np.einsum("ka,kji->aji", sz.S, rs)     # S_z^T along z
        X = np.einsum("jb,aji->abi", sy.S, X)      # S_y^T along y
        X = np.einsum("ic,abi->abc", sx.S, X)      # S_x^T along x
        X = X / (sz.lam[:, None, None] + sy.lam[None, :, None] + sx.lam[None, None, :])
        X = np.einsum("ka,abc->kbc", sz.S, X)      # S_z along z
        X = np.einsum("jb,kbc->kjc", sy.S, X)      # S_y along y
        return np.einsum("ic,kjc->kji", sx.S, X)   # S_x along x

    def schwarz_correction(self, r: np.ndarray) -> np.ndarray:
        """sum_s R_s^T W A_ss^{-1} R_s r with W = W_z (x) W_y (x) W_x."""
        du = np.zeros_like(r)
        for ez, sz in enumerate(self.dz.subs):
            for ey, sy in enumerate(self.dy.subs):
                for ex, sx in enumerate(self.dx.subs):
                    ix = np.ix_(sz.g, sy.g, sx.g)
                    w = sz.w[:, None, None] * sy.w[None, :, None] * sx.w[None, None, :]
                    du[ix] += w * self.local_solve(ex, ey, ez, r[ix])
        return du

    def wschwarz(self, u: np.ndarray, f: np.ndarray, n_it: int) -> np.ndarray:
        """Alg. 2 in 3D: n_it sweeps of weighted additive Schwarz."""
        for _ in range(n_it):
            u = u + self.schwarz_correction(f - self.apply(u))
        return u

    def dense_operator(self) -> np.ndarray:
        """Dense A over the unknowns (columns by applying A to unit vectors)."""
        idx = np.flatnonzero(self.unknown.ravel())
        A = np.zeros((len(idx), len(idx)))
        e = np.zeros(self.unknown.size)
        for c, j in enumerate(idx):
            e[j] = 1.0
            A[:, c] = self.apply(e.reshape(self.shape)).ravel()[idx]
            e[j] = 0.0
        return A


class _Coarse3:
    """Level 0 (p = 1): u_0 = A_0^+ f_0 by a dense Cholesky of A_0 (+ c 1 1^T
    when A_0 is singular, right side and solution projected; reading R7)."""

    def __init__(self, mx, my, mz):
        self.lev = Level3(mx, my, mz, 1, 0, weight="I")
        self.shape, self.unknown = self.lev.shape, self.lev.unknown
        self.idx = np.flatnonzero(self.unknown.ravel())
        A = self.lev.dense_operator()
        self.singular = self.lev.periodic
        if self.singular:
            n = len(self.idx)
            A = A + np.trace(A) / n / n * np.ones((n, n))
        self.chol = sla.cho_factor(A)

    def apply(self, u):
        return self.lev.apply(u)

    def solve(self, f):
        b = f.ravel()[self.idx]
        if self.singular:
            b = b - b.mean()
        x = sla.cho_solve(self.chol, b)
        if self.singular:
            x = x - x.mean()
        u = np.zeros(f.size)
        u[self.idx] = x
        return u.reshape(self.shape)


@dataclass
class Hierarchy3:
    """Levels p_l = 2^l, l = 0..L, in 3D, with the transfer operators."""

    mx: Mesh1D
    my: Mesh1D
    mz: Mesh1D
    p: int
    overlap: object = 1
    weight: object = 5
    levels: list = field(default_factory=list)

    def __post_init__(self):
        L = int(round(math.log2(self.p)))
        if 2**L != self.p:
            raise ValueError("p must be a power of two")
        self.L = L
        self.levels = [_Coarse3(self.mx, self.my, self.mz)]
        for l in range(1, L + 1):
            pl = 2**l
            self.levels.append(Level3(self.mx, self.my, self.mz, pl, overlap_rule(self.overlap, pl), self.weight))
        self.P = [None] + [tuple(prolongation_1d(m, 2**l, 2**(l - 1)).toarray() for m in (self.mx, self.my, self.mz))
                           for l in range(1, L + 1)]

    @property
    def top(self) -> Level3:
        return self.levels[-1]

    def prolong(self, l: int, uc: np.ndarray) -> np.ndarray:
        """I_l u_{l-1} = (P_z (x) P_y (x) P_x) u_{l-1}."""
        Px, Py, Pz = self.P[l]
        u = np.einsum("XI,KJI->KJX", Px, uc)
        u = np.einsum("YJ,KJX->KYX", Py, u)
        return np.einsum("ZK,KYX->ZYX", Pz, u)

    def restrict(self, l: int, rf: np.ndarray) -> np.ndarray:
        """I_l^T r_l; coarse wall entries are not unknowns."""
        Px, Py, Pz = self.P[l]
        rc = np.einsum("XI,ZYX->ZYI", Px, rf)
        rc = np.einsum("YJ,ZYI->ZJI", Py, rc)
        rc = np.einsum("ZK,ZJI->KJI", Pz, rc)
        return np.where(self.levels[l - 1].unknown, rc, 0.0)

    def vcycle(self, u: np.ndarray, f: np.ndarray, ns1: int = 1, ns2: int = 0) -> np.ndarray:
        """Alg. 3 with Alg. 2 as the smoother; u_l = 0 on levels l < L (R8)."""
        L = self.L
        us, fs = [None] * (L + 1), [None] * (L + 1)
        us[L], fs[L] = u, f
        for l in range(L, 0, -1):
            if l < L:
                us[l] = np.zeros_like(fs[l])
            if ns1 > 0:
                us[l] = self.levels[l].wschwarz(us[l], fs[l], ns1)
            fs[l - 1] = self.restrict(l, fs[l] - self.levels[l].apply(us[l]))
        us[0] = self.levels[0].solve(fs[0])
        for l in range(1, L + 1):
            us[l] = us[l] + self.prolong(l, us[l - 1])
            if ns2 > 0:
                us[l] = self.levels[l].wschwarz(us[l], fs[l], ns2)
        return us[L]

    def mgcg(self, u, f, n1=1, n2=0, tol=1e-10, i_max=200, precondition=True):
        """Alg. 4, inexact MG-preconditioned CG (reading R6); stops when
        ||r_i|| <= tol ||r_0||.  Returns (u, iterations, residual norms)."""
        A = self.top.apply
        M = (lambda r: self.vcycle(np.zeros_like(r), r, n1, n2)) if precondition else (lambda r: r.copy())
        r_old = np.zeros_like(f)
        r = f - A(u)
        p = M(r)
        delta = np.vdot(p, r)
        hist = [np.linalg.norm(r)]
        r_max = tol * hist[0]
        it = 0
        for i in range(1, i_max + 1):
            it = i
            q = A(p)
            alpha = delta / np.vdot(p, q)
            u = u + alpha * p
            r = r - alpha * q
            hist.append(np.linalg.norm(r))
            if hist[-1] <= r_max:
                break
            z = M(r)
            beta = np.vdot(z, r - r_old) / delta
            p = z + beta * p
            delta = np.vdot(z, r)
            r_old = r.copy()
        return u, it, hist


def uniform_hierarchy3(n, p, length=1.0, periodic=False, **kw) -> Hierarchy3:
    """n x n x n elements on [0, length]^3."""
    m = lambda: Mesh1D.uniform(n, length, periodic)
    return Hierarchy3(m(), m(), m(), p, **kw)

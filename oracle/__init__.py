"""FP64 CPU oracle for GP reconstruction + level-crossing probability.

TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the product package.  It shares no code
with the CUDA path.  Each function cites the passage of the paper it follows:
Eq. (1) (posterior), Sec. 4 (cell LCP, MC estimator), Sec. 5.1 (Slepian bound,
Eq. upper_bound), Algorithm 1 (octree adaptive query).

Parity pins live in tests/test_oracle_pins.py.  Functions without a pin:
  - gradient helpers (finite differences only; the paper has no gradient).
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np

from . import build as _build

SE = 0
MATERN52 = 1
EST_SOV = 0
EST_MC = 1
EST_INDEP = 2
EST_EDGE = 3
EST_SOV_ORD = 4

_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")


class _Grid(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("n", C.c_int64 * 3)]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        L.or_model_create.restype = C.c_void_p
        L.or_model_create.argtypes = [_dp, _dp, C.c_int64, C.c_int, _dp, C.c_double, C.c_double]
        L.or_model_destroy.argtypes = [C.c_void_p]
        L.or_model_create_sgpr.restype = C.c_void_p
        L.or_model_create_sgpr.argtypes = [_dp, _dp, _dp, C.c_int64, C.c_int, _dp, C.c_double, C.c_double]
        L.or_model_get.argtypes = [C.c_void_p] + [C.c_void_p] * 5
        L.or_kernel_eval.restype = C.c_double
        L.or_kernel_eval.argtypes = [C.c_int, _dp, C.c_double, _dp, _dp]
        L.or_cholesky.restype = C.c_int
        L.or_cholesky.argtypes = [_dp, C.c_int64]
        L.or_posterior.argtypes = [C.c_void_p, _dp, C.c_int64, _dp, _dp, C.c_void_p]
        L.or_posterior_sgpr.restype = C.c_int
        L.or_posterior_sgpr.argtypes = [C.c_void_p, _dp, _dp, _dp, C.c_int64, _dp, _dp]
        L.or_norm_cdf.restype = C.c_double
        L.or_norm_cdf.argtypes = [C.c_double]
        L.or_norm_ppf.restype = C.c_double
        L.or_norm_ppf.argtypes = [C.c_double]
        L.or_splitmix64.restype = C.c_uint64
        L.or_splitmix64.argtypes = [C.c_uint64, C.c_uint64]
        L.or_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
        L.or_sov_orthant.restype = C.c_double
        L.or_sov_orthant.argtypes = [C.c_int, _dp, _dp, C.c_int64, _u32p]
        L.or_cell_lcp.restype = C.c_double
        L.or_cell_lcp.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_int, C.c_int64, C.c_uint64,
                                  C.c_uint64, C.c_double, C.c_double]
        L.or_stats15_block.argtypes = [C.c_void_p, C.POINTER(_Grid), _i64p, _i64p, _dp]
        L.or_lcp_block.argtypes = [C.c_void_p, C.POINTER(_Grid), C.c_double, C.c_int, C.c_int64,
                                   C.c_uint64, C.c_double, C.c_double, _i64p, _i64p, _dp]
        L.or_octree_level.argtypes = [C.c_void_p, C.POINTER(_Grid), C.c_int, C.c_int, C.c_int, C.c_double,
                                      C.c_double, C.c_int, C.c_double, _i64p, C.c_int64, _i8p, _dp, _i8p]
        L.or_eval_g.argtypes = [C.c_void_p, _dp, C.c_int64, C.c_double, C.c_int, _dp, _dp]
        L.or_node_min.restype = C.c_double
        L.or_node_min.argtypes = [C.c_void_p, C.POINTER(_Grid), C.c_int, C.c_int, C.c_int, C.c_int64, C.c_double,
                                  C.c_int, C.c_int, _dp, _dp, _dp]
        L.or_bvn_lower.restype = C.c_double
        L.or_bvn_lower.argtypes = [C.c_double, C.c_double, C.c_double]
        L.or_num_threads.restype = C.c_int
        L.or_cell_lcp_adj.restype = C.c_double
        L.or_cell_lcp_adj.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_int64, C.c_uint64, C.c_uint64, C.c_double,
                                      C.c_double, C.c_double, _dp, _dp]
        L.or_cell_lcp_adj_ordered.restype = C.c_double
        L.or_cell_lcp_adj_ordered.argtypes = L.or_cell_lcp_adj.argtypes
        L.or_lcp_grad_block.restype = C.c_double
        L.or_lcp_grad_block.argtypes = [C.c_void_p, C.POINTER(_Grid), C.c_double, C.c_int64, C.c_uint64, C.c_double,
                                        C.c_double, _dp, _i64p, _i64p, _dp, _dp]
        _lib = L
    return _lib


def num_threads() -> int:
    return lib().or_num_threads()


def kernel(kind, ell, sf2, a, b) -> float:
    """k(a, b): RBF (Sec. 3) with per-axis lengths, or Matern-5/2."""
    return lib().or_kernel_eval(int(kind), np.ascontiguousarray(ell, np.float64), float(sf2),
                                np.ascontiguousarray(a, np.float64), np.ascontiguousarray(b, np.float64))


def norm_cdf(x: float) -> float:
    return lib().or_norm_cdf(float(x))


def bvn_lower(a: float, b: float, r: float) -> float:
    """P(X1 < a, X2 < b) of a standard bivariate normal with correlation r (the edge-crossing
    probability's building block, Sec. 4's line-segment formula)."""
    return lib().or_bvn_lower(float(a), float(b), float(r))


def norm_ppf(p: float) -> float:
    return lib().or_norm_ppf(float(p))


def splitmix64(seed: int, k: int) -> int:
    return int(lib().or_splitmix64(C.c_uint64(seed), C.c_uint64(k)))


def philox4x32_10(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def grid(n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)) -> _Grid:
    if np.isscalar(n):
        n = (n, n, n)
    g = _Grid()
    for d in range(3):
        g.lo[d], g.hi[d], g.n[d] = float(lo[d]), float(hi[d]), int(n[d])
    return g


class Model:
    """Plain GPR model (Sec. 3 / Eq. 1 with the observations as inducing set)."""

    def __init__(self, X, y, kernel_kind=SE, ell=(0.2, 0.2, 0.2), sf2=1.0, sn2=1e-4):
        X = np.ascontiguousarray(X, np.float64)
        y = np.ascontiguousarray(y, np.float64)
        self.m = int(y.shape[0])
        self.kernel, self.ell, self.sf2, self.sn2 = int(kernel_kind), tuple(float(e) for e in ell), float(sf2), float(sn2)
        self.X, self.y = X, y
        self._h = lib().or_model_create(X, y, self.m, self.kernel, np.asarray(self.ell, np.float64),
                                        self.sf2, self.sn2)
        if not self._h:
            raise ValueError("K(X,X) + sn2 I is not positive definite")

    @classmethod
    def from_workload(cls, w):
        if "A_M" in w.extra:
            return cls.sgpr(w.X, w.y, w.extra["A_M"], w.kernel, w.ell, w.sf2, w.extra["kmm_jitter"])
        return cls(w.X, w.y, w.kernel, w.ell, w.sf2, w.sn2)

    @classmethod
    def sgpr(cls, X, mu_M, A_M, kernel_kind=SE, ell=(0.2, 0.2, 0.2), sf2=1.0, jitter=0.0):
        """SGPR model (Sec. 3): inducing sites X with the stored distribution N(mu_M, A_M); the
        posterior is Eq. 1 as printed, with K_MM = K(X, X) + jitter I."""
        self = cls.__new__(cls)
        X = np.ascontiguousarray(X, np.float64)
        mu_M = np.ascontiguousarray(mu_M, np.float64)
        A_M = np.ascontiguousarray(A_M, np.float64)
        self.m = int(mu_M.shape[0])
        self.kernel, self.ell, self.sf2, self.sn2 = int(kernel_kind), tuple(float(e) for e in ell), float(sf2), 0.0
        self.X, self.y = X, mu_M
        self._h = lib().or_model_create_sgpr(X, mu_M, A_M.reshape(-1), self.m, self.kernel,
                                             np.asarray(self.ell, np.float64), self.sf2, float(jitter))
        if not self._h:
            raise ValueError("K_MM + jitter I is not positive definite")
        return self

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_model_destroy(h)
            self._h = None

    def factors(self):
        """Cholesky factor (of Kt, or of K_MM + jitter I for an SGPR model), alpha, L^-1 y (or
        L^-1 mu_M), and the p-test's per-observation mean and variance."""
        m = self.m
        L = np.zeros((m, m)); a = np.zeros(m); vy = np.zeros(m); mo = np.zeros(m); vo = np.zeros(m)
        lib().or_model_get(self._h, L.ctypes.data, a.ctypes.data, vy.ctypes.data, mo.ctypes.data, vo.ctypes.data)
        return {"L": L, "alpha": a, "vy": vy, "mu_obs": mo, "var_obs": vo}

    def posterior(self, P, full_cov=False):
        """Eq. (1) for plain GPR: mean, variance (and full covariance) at points P."""
        P = np.ascontiguousarray(P, np.float64).reshape(-1, 3)
        n = P.shape[0]
        mu = np.zeros(n); var = np.zeros(n)
        cov = np.zeros((n, n)) if full_cov else None
        lib().or_posterior(self._h, P, n, mu, var, cov.ctypes.data if full_cov else None)
        return (mu, var, cov) if full_cov else (mu, var)

    def posterior_sgpr(self, muM, AM, P):
        """Eq. (1) exactly as printed, for a given inducing distribution N(mu_M, A_M)."""
        P = np.ascontiguousarray(P, np.float64).reshape(-1, 3)
        n = P.shape[0]
        mu = np.zeros(n); cov = np.zeros((n, n))
        rc = lib().or_posterior_sgpr(self._h, np.ascontiguousarray(muM, np.float64),
                                     np.ascontiguousarray(AM, np.float64), P, n, mu, cov)
        if rc != 0:
            raise ValueError("K_MM not positive definite")
        return mu, cov

    def stats15(self, n, i0=(0, 0, 0), i1=None, lo=(0, 0, 0), hi=(1, 1, 1)):
        """Per-point (mu, var, 13 forward covariances) for grid points in [i0, i1)."""
        g = grid(n, lo, hi)
        if i1 is None:
            i1 = tuple(g.n)
        i0 = np.asarray(i0, np.int64); i1 = np.asarray(i1, np.int64)
        cnt = int(np.prod(i1 - i0))
        out = np.zeros(cnt * 15)
        lib().or_stats15_block(self._h, C.byref(g), i0, i1, out)
        return out.reshape(cnt, 15)

    def lcp_block(self, n, theta, c0=(0, 0, 0), c1=None, est=EST_SOV, n_samples=1600, seed=0,
                  tau=1e-10, skip_eps=1e-9, lo=(0, 0, 0), hi=(1, 1, 1)):
        """Cell LCP (Sec. 4) for cells with min corner in [c0, c1), x-fastest."""
        g = grid(n, lo, hi)
        if c1 is None:
            c1 = tuple(int(v) - 1 for v in g.n)
        c0 = np.asarray(c0, np.int64); c1 = np.asarray(c1, np.int64)
        cnt = int(np.prod(c1 - c0))
        out = np.zeros(cnt)
        lib().or_lcp_block(self._h, C.byref(g), float(theta), int(est), int(n_samples), C.c_uint64(seed),
                           float(tau), float(skip_eps), c0, c1, out)
        return out

    def lcp_dense(self, n, theta, slab=8, **kw):
        """Dense baseline LCP field (Sec. 4 / Sec. 6.4), computed in z-slabs."""
        nc = n - 1
        out = np.zeros(nc ** 3)
        for z0 in range(0, nc, slab):
            z1 = min(nc, z0 + slab)
            out[z0 * nc * nc: z1 * nc * nc] = self.lcp_block(n, theta, (0, 0, z0), (nc, nc, z1), **kw)
        return out

    def octree_level(self, n, D, l, theta, nodes, alpha=1e-3, T=4, beta=-1.0, kd=False):
        """One level of Algorithm 1.  Returns (decision, bound, side) per node.  beta >= 0: the
        bound uses each node's local model (Sec. 5.2, beta in length scales); beta < 0: the full one.
        kd: level l (0 .. 3D) of the K-D tree of Sec. 9 instead of the octree."""
        g = grid(n)
        nodes = np.ascontiguousarray(nodes, np.int64)
        cnt = nodes.shape[0]
        dec = np.zeros(cnt, np.int8); bnd = np.zeros(cnt); side = np.zeros(cnt, np.int8)
        if cnt:
            lib().or_octree_level(self._h, C.byref(g), int(D), int(l), int(bool(kd)), float(theta), float(alpha),
                                  int(T), float(beta), nodes, cnt, dec, bnd, side)
        return dec, bnd, side

    def octree(self, n, D, theta, alpha=1e-3, T=4, beta=-1.0, kd=False):
        """Algorithm 1 top-down, level by level (D + 1 octree levels, or 3D + 1 levels of the K-D tree
        of Sec. 9, which halves x, y, z in turn).  Returns (S cell codes, per-level records)."""
        nodes = np.zeros(1, np.int64)
        levels = []
        leaves = np.zeros(0, np.int64)
        last = 3 * D if kd else D
        for l in range(last + 1):
            dec, bnd, side = self.octree_level(n, D, l, theta, nodes, alpha, T, beta, kd)
            levels.append({"nodes": nodes, "decision": dec, "bound": bnd, "side": side})
            keep = nodes[dec > 0]
            if l == last:
                leaves = keep
                break
            i = keep & 0x1FFFFF; j = (keep >> 21) & 0x1FFFFF; k = (keep >> 42) & 0x1FFFFF
            ch = []
            if kd:
                a = l % 3  # the axis this level halves
                s_child = [1 << (D - (l + 1 + 2 - d) // 3) for d in range(3)]
                for b in range(2):
                    c3 = [i, j, k]
                    c3[a] = 2 * c3[a] + b
                    ok = (c3[0] * s_child[0] < n - 1) & (c3[1] * s_child[1] < n - 1) & (c3[2] * s_child[2] < n - 1)
                    ch.append((c3[0] | (c3[1] << 21) | (c3[2] << 42))[ok])
            else:
                s_child = 1 << (D - l - 1)
                for c in range(8):
                    ci = 2 * i + (c & 1); cj = 2 * j + ((c >> 1) & 1); ck = 2 * k + ((c >> 2) & 1)
                    ok = (ci * s_child < n - 1) & (cj * s_child < n - 1) & (ck * s_child < n - 1)
                    ch.append((ci | (cj << 21) | (ck << 42))[ok])
            nodes = np.sort(np.concatenate(ch)) if ch else np.zeros(0, np.int64)
        return leaves, levels

    def lcp_adaptive(self, n, D, theta, alpha=1e-3, T=4, beta=-1.0, kd=False, **kw):
        """Adaptive LCP field: the dense cell LCP on the leaves S of Algorithm 1, 0 elsewhere (Sec. 5.3)."""
        leaves, levels = self.octree(n, D, theta, alpha, T, beta, kd)
        nc = n - 1
        field = np.zeros(nc ** 3)
        if leaves.size:
            ci = leaves & 0x1FFFFF; cj = (leaves >> 21) & 0x1FFFFF; ck = (leaves >> 42) & 0x1FFFFF
            lin = ci + nc * (cj + nc * ck)
            dense = self.lcp_dense(n, theta, **kw)
            field[lin] = dense[lin]
        return field, leaves, levels

    def lcp_grad(self, n, theta, weights, c0=(0, 0, 0), c1=None, n_samples=1600, seed=0, tau=1e-10, skip_eps=1e-9):
        """Gradient of sum_c weights[c] LCP_c over cells [c0, c1) wrt y and log length scales;
        `weights` is indexed by the linear cell index of the whole grid (one per grid cell).
        Returns (loss, dL/dy, dL/dlog l)."""
        weights = np.ascontiguousarray(weights, np.float64)
        if weights.size != int(np.prod([v - 1 for v in (n, n, n)])):
            raise ValueError("lcp_grad: one weight per cell of the whole grid")
        g = grid(n)
        if c1 is None:
            c1 = tuple(int(v) - 1 for v in g.n)
        c0 = np.asarray(c0, np.int64); c1 = np.asarray(c1, np.int64)
        dy = np.zeros(self.m); dl = np.zeros(3)
        loss = lib().or_lcp_grad_block(self._h, C.byref(g), float(theta), int(n_samples), C.c_uint64(seed), float(tau),
                                       float(skip_eps), np.ascontiguousarray(weights, np.float64), c0, c1, dy, dl)
        return loss, dy, dl

    def node_min(self, n, D, l, node, theta, side, T=4, kd=False):
        """The node minimiser of Algorithm 1's bound (Sec. 5.1) for one node and one side:
        (min g, the point where it was found, box lo, box hi), g = side*(theta-mu)/sigma."""
        g = grid(n)
        x = np.zeros(3); lo = np.zeros(3); hi = np.zeros(3)
        v = lib().or_node_min(self._h, C.byref(g), int(D), int(l), int(bool(kd)), int(node), float(theta), int(side),
                              int(T), x, lo, hi)
        return v, x, lo, hi

    def eval_g(self, x, theta, side):
        x = np.ascontiguousarray(x, np.float64).reshape(-1, 3)
        g = np.zeros(x.shape[0]); gr = np.zeros((x.shape[0], 3))
        lib().or_eval_g(self._h, x, x.shape[0], float(theta), int(side), g, gr.reshape(-1))
        return g, gr


def cell_lcp_adj(mu, S, theta, wbar=1.0, n_samples=1600, seed=0, cell=0, tau=1e-10, skip_eps=1e-9, est=EST_SOV):
    """Adjoint of the SOV cell rule (est EST_SOV, or EST_SOV_ORD for the ordered rule):
    (LCP, dLCP/dmu * wbar, dLCP/dSigma * wbar)."""
    mu = np.ascontiguousarray(mu, np.float64)
    S = np.ascontiguousarray(S, np.float64)
    d = mu.shape[0]
    mb = np.zeros(d); Sb = np.zeros(d * d)
    fn = lib().or_cell_lcp_adj_ordered if est == EST_SOV_ORD else lib().or_cell_lcp_adj
    v = fn(d, mu, S.reshape(-1), float(theta), int(n_samples), C.c_uint64(seed), C.c_uint64(cell),
           float(tau), float(skip_eps), float(wbar), mb, Sb)
    return v, mb, Sb.reshape(d, d)


def cell_lcp(mu, S, theta, est=EST_SOV, n_samples=1600, seed=0, cell=0, tau=1e-10, skip_eps=1e-9):
    """LCP of one cell (or any d <= 16 corner variables) from (mu, Sigma) (Sec. 4)."""
    mu = np.ascontiguousarray(mu, np.float64)
    S = np.ascontiguousarray(S, np.float64)
    d = mu.shape[0]
    return lib().or_cell_lcp(d, mu, S.reshape(-1), float(theta), int(est), int(n_samples), C.c_uint64(seed),
                             C.c_uint64(cell), float(tau), float(skip_eps))


def sov_orthant(L, b, n_samples, shift):
    """P(X <= b), X ~ N(0, L L^T) by the sequential-conditioning lattice rule."""
    L = np.ascontiguousarray(L, np.float64)
    d = L.shape[0]
    return lib().or_sov_orthant(d, L.reshape(-1), np.ascontiguousarray(b, np.float64), int(n_samples),
                                np.ascontiguousarray(shift, np.uint32))

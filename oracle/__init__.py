"""ctypes front end of the FP64 CPU oracle (hermite_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package entry point's
smoke check and by the benchmark's CPU-baseline leg.  The product library never
imports it.  All 3-vector arrays here are numpy float64 [n, 3] (array of
structures), matching the C file.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hermite_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libhermite_oracle.so")
_lib = None

_D = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I32 = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_I64 = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_U64 = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "hermite_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


class HhoParams(C.Structure):
    _fields_ = [("eps2", C.c_double), ("eta", C.c_double), ("eta_s", C.c_double),
                ("dt_min", C.c_double), ("dt_max", C.c_double), ("dt_tree", C.c_double),
                ("theta", C.c_double), ("leaf", C.c_int), ("n_crit", C.c_int), ("use_tree", C.c_int)]


class HhoStats(C.Structure):
    _fields_ = [("block_steps", C.c_int64), ("particle_steps", C.c_int64),
                ("interactions", C.c_int64), ("rebuilds", C.c_int64)]


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.hho_direct_force.argtypes = [C.c_int, _D, _D, _D, C.c_double, _D, _D, _D]
        L.hho_direct_force_subset.argtypes = [C.c_int, _D, _D, _D, C.c_double, C.c_int, _I32, _D, _D, _D]
        L.hho_list_force.argtypes = [C.c_int, _D, _D, _D, C.c_int, _I32, _I32, _I64, _I32, C.c_double,
                                     _D, _D, _D]
        L.hho_predict.argtypes = [C.c_int, _D, _D, _D, _D, _D, C.c_double, _D, _D]
        L.hho_correct_one.argtypes = [C.c_double, _D, _D, _D, _D, _D, _D, _D, _D, _D, _D]
        L.hho_aarseth_dt.argtypes = [C.c_double, _D, _D, _D, _D]
        L.hho_aarseth_dt.restype = C.c_double
        L.hho_block_dt.argtypes = [C.c_double] * 5
        L.hho_block_dt.restype = C.c_double
        L.hho_initial_dt.argtypes = [C.c_double, _D, _D, C.c_double, C.c_double]
        L.hho_initial_dt.restype = C.c_double
        L.hho_tree_build.argtypes = [C.c_int, _D, _D, _D, _D, _D, C.c_int, C.c_int, C.c_double]
        L.hho_tree_build.restype = C.c_void_p
        L.hho_tree_build_ordered.argtypes = [C.c_int, _D, _D, _D, _D, _D, C.c_int, C.c_int, C.c_double, C.c_int]
        L.hho_tree_build_ordered.restype = C.c_void_p
        L.hho_morton_key.argtypes = [C.c_uint32] * 3
        L.hho_morton_key.restype = C.c_uint64
        L.hho_hilbert_key.argtypes = [C.c_uint32] * 3 + [C.c_int]
        L.hho_hilbert_key.restype = C.c_uint64
        L.hho_tree_free.argtypes = [C.c_void_p]
        for f in ("hho_tree_n_cells", "hho_tree_n_groups"):
            getattr(L, f).argtypes = [C.c_void_p]
            getattr(L, f).restype = C.c_int
        L.hho_tree_list_len.argtypes = [C.c_void_p]
        L.hho_tree_list_len.restype = C.c_int64
        L.hho_tree_perm.argtypes = [C.c_void_p, _I32]
        L.hho_tree_keys.argtypes = [C.c_void_p, _U64]
        L.hho_tree_nodes.argtypes = [C.c_void_p, _D, _D, _D, _D, _D]
        L.hho_tree_cells.argtypes = [C.c_void_p, _I32, _I32, _I32, _D]
        L.hho_tree_groups.argtypes = [C.c_void_p, _I32, _I32, _I32, _I32]
        L.hho_tree_lists.argtypes = [C.c_void_p, _I64, _I32]
        L.hho_run.argtypes = [C.c_int, _D, _D, _D, C.c_double, C.POINTER(HhoParams), _D, _D, _D, _D,
                              C.POINTER(HhoStats)]
        L.hho_run.restype = C.c_int
        L.hho_resume.argtypes = [C.c_int, _D, _D, _D, _D, _D, _D, C.c_double, C.c_double, C.POINTER(HhoParams),
                                 C.POINTER(HhoStats)]
        L.hho_resume.restype = C.c_int
        L.hho_energy.argtypes = [C.c_int, _D, _D, _D, C.c_double]
        L.hho_energy.restype = C.c_double
        L.hho_num_threads.restype = C.c_int
        _lib = L
    return _lib


def _v3(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None:
        assert a.shape == (n, 3), a.shape
    return a


def num_threads() -> int:
    return lib().hho_num_threads()


def direct_force(x, v, m, eps2):
    """Direct softened sum over all other particles: (acc[n,3], jerk[n,3], pot[n])."""
    n = len(m)
    x, v, m = _v3(x, n), _v3(v, n), np.ascontiguousarray(m, dtype=np.float64)
    acc, jerk, pot = np.zeros((n, 3)), np.zeros((n, 3)), np.zeros(n)
    lib().hho_direct_force(n, x, v, m, float(eps2), acc, jerk, pot)
    return acc, jerk, pot


def direct_force_subset(x, v, m, eps2, i_idx):
    n = len(m)
    x, v, m = _v3(x, n), _v3(v, n), np.ascontiguousarray(m, dtype=np.float64)
    i_idx = np.ascontiguousarray(i_idx, dtype=np.int32)
    k = len(i_idx)
    acc, jerk, pot = np.zeros((k, 3)), np.zeros((k, 3)), np.zeros(k)
    lib().hho_direct_force_subset(n, x, v, m, float(eps2), k, i_idx, acc, jerk, pot)
    return acc, jerk, pot


def list_force(xj, vj, mj, i_idx, gid, list_off, list_idx, eps2):
    """Force on active j-array particles i_idx (group ids gid) from their lists."""
    nj = len(mj)
    xj, vj, mj = _v3(xj, nj), _v3(vj, nj), np.ascontiguousarray(mj, dtype=np.float64)
    i_idx = np.ascontiguousarray(i_idx, dtype=np.int32)
    gid = np.ascontiguousarray(gid, dtype=np.int32)
    k = len(i_idx)
    acc, jerk, pot = np.zeros((k, 3)), np.zeros((k, 3)), np.zeros(k)
    lib().hho_list_force(nj, xj, vj, mj, k, i_idx, gid, np.ascontiguousarray(list_off, dtype=np.int64),
                         np.ascontiguousarray(list_idx, dtype=np.int32), float(eps2), acc, jerk, pot)
    return acc, jerk, pot


def predict(x, v, a, jk, t0, t):
    n = len(t0)
    xp, vp = np.zeros((n, 3)), np.zeros((n, 3))
    lib().hho_predict(n, _v3(x, n), _v3(v, n), _v3(a, n), _v3(jk, n),
                      np.ascontiguousarray(t0, dtype=np.float64), float(t), xp, vp)
    return xp, vp


def correct_one(dt, xp, vp, a0, j0, a1, j1):
    out = [np.zeros(3) for _ in range(4)]
    args = [np.ascontiguousarray(u, dtype=np.float64) for u in (xp, vp, a0, j0, a1, j1)]
    lib().hho_correct_one(float(dt), *args, *out)
    return tuple(out)  # x1, v1, a2_end, a3


def aarseth_dt(eta, a, j, a2, a3):
    return lib().hho_aarseth_dt(float(eta), *[np.ascontiguousarray(u, dtype=np.float64) for u in (a, j, a2, a3)])


def block_dt(dt_want, dt_old, t_new, dt_min, dt_max):
    return lib().hho_block_dt(float(dt_want), float(dt_old), float(t_new), float(dt_min), float(dt_max))


def initial_dt(eta_s, a, j, dt_min, dt_max):
    return lib().hho_initial_dt(float(eta_s), np.ascontiguousarray(a, dtype=np.float64),
                                np.ascontiguousarray(j, dtype=np.float64), float(dt_min), float(dt_max))


@dataclass
class Tree:
    """Morton octree, groups and lists built by the oracle.

    perm[k]: input index of Morton position k.  Node k (cell k) has j-index n+k.
    """
    n: int
    perm: np.ndarray
    keys: np.ndarray
    node_x: np.ndarray
    node_v: np.ndarray
    node_a: np.ndarray
    node_j: np.ndarray
    node_m: np.ndarray
    cell_begin: np.ndarray
    cell_end: np.ndarray
    cell_depth: np.ndarray
    cell_side: np.ndarray
    g_cell: np.ndarray
    g_begin: np.ndarray
    g_end: np.ndarray
    group_of: np.ndarray
    list_off: np.ndarray
    list_idx: np.ndarray

    @property
    def n_cells(self):
        return len(self.node_m)

    @property
    def n_groups(self):
        return len(self.g_cell)

    def j_array(self, x, v, a, jk, m):
        """Particles (input order arrays) in Morton order followed by the node records."""
        p = self.perm
        cat = lambda u, nd: np.concatenate([np.asarray(u, dtype=np.float64)[p], nd])
        return (cat(x, self.node_x), cat(v, self.node_v), cat(a, self.node_a), cat(jk, self.node_j),
                cat(m, self.node_m))


def morton_key(ix, iy, iz):
    return int(lib().hho_morton_key(int(ix), int(iy), int(iz)))


def hilbert_key(ix, iy, iz, bits):
    """Peano-Hilbert index of cell (ix, iy, iz) of a 2^bits grid (Section 2's order)."""
    return int(lib().hho_hilbert_key(int(ix), int(iy), int(iz), int(bits)))


ORDERS = {"morton": 0, "hilbert": 1}


def tree_build(x, v, a, jk, m, leaf=8, n_crit=64, theta=0.5, order="morton") -> Tree:
    n = len(m)
    L = lib()
    h = L.hho_tree_build_ordered(n, _v3(x, n), _v3(v, n), _v3(a, n), _v3(jk, n),
                                 np.ascontiguousarray(m, dtype=np.float64), int(leaf), int(n_crit), float(theta),
                                 ORDERS[order])
    if not h:
        raise ValueError("hho_tree_build failed")
    try:
        nc, ng, ll = L.hho_tree_n_cells(h), L.hho_tree_n_groups(h), L.hho_tree_list_len(h)
        perm = np.zeros(n, np.int32)
        keys = np.zeros(n, np.uint64)
        L.hho_tree_perm(h, perm)
        L.hho_tree_keys(h, keys)
        nx, nv, na, nj = (np.zeros((nc, 3)) for _ in range(4))
        nm = np.zeros(nc)
        L.hho_tree_nodes(h, nx, nv, na, nj, nm)
        cb, ce, cd = (np.zeros(nc, np.int32) for _ in range(3))
        cs = np.zeros(nc)
        L.hho_tree_cells(h, cb, ce, cd, cs)
        gc, gb, ge = (np.zeros(ng, np.int32) for _ in range(3))
        gof = np.zeros(n, np.int32)
        L.hho_tree_groups(h, gc, gb, ge, gof)
        off = np.zeros(ng + 1, np.int64)
        idx = np.zeros(max(ll, 1), np.int32)
        L.hho_tree_lists(h, off, idx)
        idx = idx[:ll]
    finally:
        L.hho_tree_free(h)
    return Tree(n, perm, keys, nx, nv, na, nj, nm, cb, ce, cd, cs, gc, gb, ge, gof, off, idx)


@dataclass
class RunParams:
    eps2: float = 1e-8
    eta: float = 0.02
    eta_s: float = 0.01
    dt_min: float = 2.0 ** -30
    dt_max: float = 2.0 ** -6
    dt_tree: float = 2.0 ** -6
    theta: float = 0.5
    leaf: int = 8
    n_crit: int = 64
    use_tree: bool = True

    def c(self):
        return HhoParams(self.eps2, self.eta, self.eta_s, self.dt_min, self.dt_max, self.dt_tree,
                         self.theta, self.leaf, self.n_crit, int(self.use_tree))


def run(x, v, m, t_end, params: RunParams):
    """Hermite block-step integration; returns dict(x, v, a, jk, t, dt, stats)."""
    n = len(m)
    x = _v3(x, n).copy()
    v = _v3(v, n).copy()
    a, jk = np.zeros((n, 3)), np.zeros((n, 3))
    t, dt = np.zeros(n), np.zeros(n)
    st = HhoStats()
    cp = params.c()
    rc = lib().hho_run(n, x, v, np.ascontiguousarray(m, dtype=np.float64), float(t_end), C.byref(cp),
                       a, jk, t, dt, C.byref(st))
    if rc != 0:
        raise RuntimeError(f"hho_run failed: {rc}")
    return dict(x=x, v=v, a=a, jk=jk, t=t, dt=dt,
                stats=dict(block_steps=st.block_steps, particle_steps=st.particle_steps,
                           interactions=st.interactions, rebuilds=st.rebuilds))


def resume(x, v, a, jk, dt, m, t0, t_end, params: RunParams):
    """The run continued from a synchronised state at t0 (a multiple of
    dt_tree): x, v, a, jk [n, 3] and dt [n] of every particle at t0.  Returns
    dict(x, v, a, jk, dt, stats) at t_end; the inputs are not modified."""
    n = len(m)
    x, v, a, jk = (_v3(u, n).copy() for u in (x, v, a, jk))
    dt = np.ascontiguousarray(dt, dtype=np.float64).copy()
    st = HhoStats()
    cp = params.c()
    rc = lib().hho_resume(n, x, v, a, jk, dt, np.ascontiguousarray(m, dtype=np.float64), float(t0), float(t_end),
                          C.byref(cp), C.byref(st))
    if rc != 0:
        raise RuntimeError(f"hho_resume failed: {rc}")
    return dict(x=x, v=v, a=a, jk=jk, dt=dt,
                stats=dict(block_steps=st.block_steps, particle_steps=st.particle_steps,
                           interactions=st.interactions, rebuilds=st.rebuilds))


def energy(x, v, m, eps2):
    n = len(m)
    return lib().hho_energy(n, _v3(x, n), _v3(v, n), np.ascontiguousarray(m, dtype=np.float64), float(eps2))

"""Python binding of libhh: the list-driven 4th-order Hermite force path on GB300.

Argument marshalling only.  Every step of the path runs in libhh's CUDA
kernels (or, for the tree builder, its native host code); there is no Python or
CPU fallback: importing this package raises if libhh.so has not been built.

Functions keep the C names (see include/hh.h).  Host arrays are numpy float64
arrays in structure-of-arrays layout [3, n] for 3-vectors; the *_dev calls take
torch CUDA tensors (or raw device pointers) and run on the context's stream.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhh.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libhh.so is not built ({LIB_PATH}); run paper_1602_02832_gb300/build.py "
                      "or __graft_entry__.build() first")

_lib = C.CDLL(LIB_PATH)

HH_OK, HH_EINVAL, HH_ENOMEM, HH_ECUDA, HH_ETIMEOUT, HH_ESTATE = 0, -1, -2, -3, -4, -5
HH_FP64, HH_MIXED = 0, 1
HH_ORDER_MORTON, HH_ORDER_HILBERT = 0, 1
_ERR_NAMES = {HH_EINVAL: "HH_EINVAL", HH_ENOMEM: "HH_ENOMEM", HH_ECUDA: "HH_ECUDA", HH_ETIMEOUT: "HH_ETIMEOUT",
              HH_ESTATE: "HH_ESTATE"}


class HHError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


class hh_config(C.Structure):
    _fields_ = [("eps2", C.c_double), ("eta", C.c_double), ("eta_s", C.c_double), ("dt_min", C.c_double),
                ("dt_max", C.c_double), ("dt_tree", C.c_double), ("theta", C.c_double), ("leaf", C.c_int32),
                ("n_crit", C.c_int32), ("precision", C.c_int32), ("tile_i", C.c_int32), ("tile_j", C.c_int32),
                ("work_item", C.c_int32), ("order", C.c_int32), ("work_split", C.c_int32),
                ("tile_j_small", C.c_int32)]


class hh_counters(C.Structure):
    _fields_ = [("block_steps", C.c_int64), ("particle_steps", C.c_int64), ("interactions", C.c_int64),
                ("rebuilds", C.c_int64), ("tile_steps", C.c_int64), ("list_steps", C.c_int64)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I32 = C.POINTER(C.c_int32)
_I64 = C.POINTER(C.c_int64)

_SIGS = {
    "hh_config_default": (None, [C.POINTER(hh_config)]),
    "hh_create": (C.c_int, [C.POINTER(_P), C.c_int, C.POINTER(hh_config), C.c_int64, C.c_int64, C.c_int64,
                            C.c_int32]),
    "hh_destroy": (C.c_int, [_P]),
    "hh_set_stream": (C.c_int, [_P, _P]),
    "hh_set_j": (C.c_int, [_P, C.c_int64, C.c_int64, _D, _D, _D, _D, _D, _D]),
    "hh_set_j_dev": (C.c_int, [_P, C.c_int64, C.c_int64, _P, _P, _P, _P, _P, _P]),
    "hh_set_lists": (C.c_int, [_P, C.c_int64, C.c_int64, C.c_int32, _I64, _I32, _I32]),
    "hh_set_dt": (C.c_int, [_P, _D]),
    "hh_init_dt": (C.c_int, [_P]),
    "hh_predict": (C.c_int, [_P, C.c_double]),
    "hh_force": (C.c_int, [_P, C.c_int32, _I32, _D, _D, _D]),
    "hh_force_dev": (C.c_int, [_P, C.c_int32, _P, _P, _P, _P]),
    "hh_correct": (C.c_int, [_P, C.c_double, C.c_int32, _I32]),
    "hh_init_forces": (C.c_int, [_P, C.c_double]),
    "hh_step": (C.c_int, [_P, _D, _I32]),
    "hh_advance": (C.c_int, [_P, C.c_double, _I64]),
    "hh_rebuild": (C.c_int, [_P, C.c_double]),
    "hh_load_particles": (C.c_int, [_P, C.c_int64, _D, _D, _D, C.c_double]),
    "hh_run": (C.c_int, [_P, C.c_double, C.c_double]),
    "hh_get_state": (C.c_int, [_P, _D, _D, _D, _D, _D, _D]),
    "hh_get_ids": (C.c_int, [_P, _I64]),
    "hh_n_particles": (C.c_int64, [_P]),
    "hh_n_j": (C.c_int64, [_P]),
    "hh_get_counters": (C.c_int, [_P, C.POINTER(hh_counters)]),
    "hh_reset_counters": (C.c_int, [_P]),
    "hh_get_tile_histogram": (C.c_int, [_P, _P]),
    "hh_force_timing": (C.c_int, [_P, C.c_int, _D, _I64]),
    "hh_kernel_launches": (C.c_int64, []),
    "hh_last_error": (C.c_char_p, [_P]),
    "hh_tree_build": (C.c_int, [C.POINTER(_P), C.c_int64, _D, _D, _D, _D, _D, C.c_int32, C.c_int32, C.c_double]),
    "hh_tree_build_ordered": (C.c_int, [C.POINTER(_P), C.c_int64, _D, _D, _D, _D, _D, C.c_int32, C.c_int32, C.c_double,
                                        C.c_int32]),
    "hh_tree_sizes": (C.c_int, [_P, _I64, _I32, _I64]),
    "hh_tree_export": (C.c_int, [_P, _I32, _D, _D, _D, _D, _D, _I64, _I32, _I32]),
    "hh_tree_free": (C.c_int, [_P]),
    "hh_force_static": (C.c_int, [C.c_int, C.c_int, C.c_double, C.c_int64, _P, _P, _P, C.c_int32, _P, _P, C.c_int32,
                                  _P, _P, _P, _P, _P, _P]),
    "hh_batch_create": (C.c_int, [C.POINTER(_P), C.c_int, C.c_int, C.c_int32, C.c_int32]),
    "hh_batch_destroy": (C.c_int, [_P]),
    "hh_batch_run": (C.c_int, [_P, C.c_int32, C.POINTER(_P), _D, C.c_int32, _I32, _D, _D, _D]),
    "hh_batch_last_error": (C.c_char_p, [_P]),
    "hh_batch_set_budget": (C.c_int, [_P, C.c_int64, C.c_int64]),
    "hh_batch_admit": (C.c_int, [_P, _P, C.c_double]),
    "hh_batch_step": (C.c_int, [_P, C.c_int32, _I32, _I32, _I32, C.POINTER(_P), _D, _D]),
    "hh_batch_retire": (C.c_int, [_P, _P]),
    "hh_batch_resident": (C.c_int, [_P, _I32, _I32, _I64]),
    "hh_batch_rebuild": (C.c_int, [_P, C.c_int32, C.POINTER(_P), _D, C.POINTER(C.c_int)]),
    "hh_ctx_device_bytes": (C.c_int64, [_P]),
    "hh_barrier_selftest": (C.c_int, [C.c_int, C.c_int, _D]),
    "hh_selftest_aarseth": (C.c_int, [C.c_int, C.c_int64, _D, _D, _D, _D, C.c_double, _D]),
    "hh_batch_set_ctas": (C.c_int, [_P, C.c_int32]),
    "hh_selftest_block_dt": (C.c_int, [C.c_int, C.c_int64, _D, _D, _D, C.c_double, C.c_double, _D]),
    "hh_set_rebuild_device": (C.c_int, [_P, C.c_int]),
    "hh_get_lists": (C.c_int, [_P, _I32, _I64, _I64, _I32, _I32]),
    "hh_get_j": (C.c_int, [_P, C.c_int64, C.c_int64, _D, _D, _D, _D, _D, _D]),
}

for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


def lib():
    return _lib


def _ptr(a, ct=C.c_double):
    return None if a is None else a.ctypes.data_as(C.POINTER(ct))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        raise ValueError(f"expected shape {shape}, got {a.shape}")
    return a


def _dev_ptr(t):
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not (t.is_cuda and t.is_contiguous()):
        raise ValueError("device arrays must be contiguous CUDA tensors")
    return t.data_ptr()


def _check(rc, ctx=None):
    if rc != HH_OK:
        msg = _lib.hh_last_error(ctx)
        raise HHError(rc, msg.decode() if msg else "")
    return rc


def hh_last_error(ctx=None) -> str:
    m = _lib.hh_last_error(ctx)
    return m.decode() if m else ""


def hh_config_default() -> hh_config:
    c = hh_config()
    _lib.hh_config_default(C.byref(c))
    return c


def hh_kernel_launches() -> int:
    return int(_lib.hh_kernel_launches())


class Context:
    """One simulation's device state (wraps an hh_ctx*)."""

    def __init__(self, cfg: hh_config | None = None, n_max: int = 1, nj_max: int = 1, list_max: int = 1,
                 groups_max: int = 1, device: int = 0):
        cfg = cfg or hh_config_default()
        h = _P()
        _check(_lib.hh_create(C.byref(h), device, C.byref(cfg), n_max, nj_max, list_max, groups_max))
        self.h = h
        self.cfg = cfg
        self.n_max, self.nj_max = n_max, nj_max

    def close(self):
        if getattr(self, "h", None):
            _lib.hh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _c(self, rc):
        return _check(rc, self.h)

    # -- step 1 -----------------------------------------------------------
    def hh_set_stream(self, stream):
        s = stream if isinstance(stream, int) else (stream.cuda_stream if stream is not None else None)
        self._c(_lib.hh_set_stream(self.h, s))

    def hh_set_j(self, first, x, v, a, jk, m, t):
        n = len(m)
        arrs = [_f64(u, (3, n)) for u in (x, v, a, jk)] + [_f64(m, (n,)), _f64(t, (n,))]
        self._c(_lib.hh_set_j(self.h, first, n, *[_ptr(u) for u in arrs]))

    def hh_set_j_dev(self, first, x, v, a, jk, m, t):
        n = m.numel() if hasattr(m, "numel") else int(m)
        self._c(_lib.hh_set_j_dev(self.h, first, n, *[_dev_ptr(u) for u in (x, v, a, jk, m, t)]))

    def hh_set_lists(self, n_particles, n_j, off, idx, group_of):
        off = np.ascontiguousarray(off, dtype=np.int64)
        idx = np.ascontiguousarray(idx, dtype=np.int32)
        if idx.size == 0:
            idx = np.zeros(1, np.int32)
        gof = np.ascontiguousarray(group_of, dtype=np.int32)
        self._c(_lib.hh_set_lists(self.h, n_particles, n_j, len(off) - 1, _ptr(off, C.c_int64),
                                  _ptr(idx, C.c_int32), _ptr(gof, C.c_int32)))

    def hh_set_dt(self, dt):
        self._c(_lib.hh_set_dt(self.h, _ptr(_f64(dt))))

    def hh_init_dt(self):
        self._c(_lib.hh_init_dt(self.h))

    # -- steps 4, 4a + 5, 6 ----------------------------------------------------
    def hh_predict(self, t):
        self._c(_lib.hh_predict(self.h, float(t)))

    def hh_force(self, i_idx, want=(True, True, True)):
        i_idx = np.ascontiguousarray(i_idx, dtype=np.int32)
        k = len(i_idx)
        acc = np.zeros((3, k)) if want[0] else None
        jerk = np.zeros((3, k)) if want[1] else None
        pot = np.zeros(k) if want[2] else None
        self._c(_lib.hh_force(self.h, k, _ptr(i_idx, C.c_int32), _ptr(acc), _ptr(jerk), _ptr(pot)))
        return acc, jerk, pot

    def hh_force_dev(self, i_idx, acc, jerk, pot):
        n = i_idx.numel()
        self._c(_lib.hh_force_dev(self.h, n, _dev_ptr(i_idx), _dev_ptr(acc), _dev_ptr(jerk), _dev_ptr(pot)))

    def hh_correct(self, t, i_idx):
        i_idx = np.ascontiguousarray(i_idx, dtype=np.int32)
        self._c(_lib.hh_correct(self.h, float(t), len(i_idx), _ptr(i_idx, C.c_int32)))

    def hh_init_forces(self, t):
        self._c(_lib.hh_init_forces(self.h, float(t)))

    # -- device-resident loop --------------------------------------------------
    def hh_step(self):
        t = C.c_double()
        na = C.c_int32()
        self._c(_lib.hh_step(self.h, C.byref(t), C.byref(na)))
        return t.value, na.value

    def hh_advance(self, t_end):
        ns = C.c_int64()
        self._c(_lib.hh_advance(self.h, float(t_end), C.byref(ns)))
        return ns.value

    def hh_rebuild(self, t):
        self._c(_lib.hh_rebuild(self.h, float(t)))

    def hh_set_rebuild_device(self, on=True):
        self._c(_lib.hh_set_rebuild_device(self.h, int(bool(on))))

    def hh_load_particles(self, x, v, m, t=0.0):
        n = len(m)
        self._c(_lib.hh_load_particles(self.h, n, _ptr(_f64(x, (3, n))), _ptr(_f64(v, (3, n))),
                                       _ptr(_f64(m, (n,))), float(t)))

    def hh_run(self, t0, t_end):
        self._c(_lib.hh_run(self.h, float(t0), float(t_end)))

    # -- readback ----------------------------------------------------------------
    @property
    def n(self):
        return int(_lib.hh_n_particles(self.h))

    @property
    def nj(self):
        return int(_lib.hh_n_j(self.h))

    def hh_get_state(self):
        n = self.n
        x, v, a, jk = (np.zeros((3, n)) for _ in range(4))
        t, dt = np.zeros(n), np.zeros(n)
        self._c(_lib.hh_get_state(self.h, *[_ptr(u) for u in (x, v, a, jk, t, dt)]))
        return dict(x=x, v=v, a=a, jk=jk, t=t, dt=dt)

    def hh_get_lists(self):
        g, L = C.c_int32(), C.c_int64()
        self._c(_lib.hh_get_lists(self.h, C.byref(g), C.byref(L), None, None, None))
        off = np.zeros(g.value + 1, np.int64)
        idx = np.zeros(max(L.value, 1), np.int32)
        gof = np.zeros(self.n, np.int32)
        self._c(_lib.hh_get_lists(self.h, None, None, _ptr(off, C.c_int64), _ptr(idx, C.c_int32),
                                  _ptr(gof, C.c_int32)))
        return off, idx[:L.value], gof

    def hh_get_j(self, first, count):
        x, v, a, jk = (np.zeros((3, count)) for _ in range(4))
        m, t = np.zeros(count), np.zeros(count)
        self._c(_lib.hh_get_j(self.h, int(first), int(count), *[_ptr(u) for u in (x, v, a, jk, m, t)]))
        return dict(x=x, v=v, a=a, jk=jk, m=m, t=t)

    def hh_get_ids(self):
        ids = np.zeros(self.n, np.int64)
        self._c(_lib.hh_get_ids(self.h, _ptr(ids, C.c_int64)))
        return ids

    def hh_get_counters(self):
        c = hh_counters()
        self._c(_lib.hh_get_counters(self.h, C.byref(c)))
        return dict(block_steps=c.block_steps, particle_steps=c.particle_steps, interactions=c.interactions,
                    rebuilds=c.rebuilds, tile_steps=c.tile_steps, list_steps=c.list_steps)

    def hh_get_tile_histogram(self):
        """counts[k] = active i tiles evaluated with k + 1 active particles."""
        h = np.zeros(32, np.int64)
        self._c(_lib.hh_get_tile_histogram(self.h, _ptr(h, C.c_int64)))
        return h

    def hh_reset_counters(self):
        self._c(_lib.hh_reset_counters(self.h))

    @property
    def device_bytes(self):
        return int(_lib.hh_ctx_device_bytes(self.h))

    def hh_force_timing(self, enable=-1):
        ms = C.c_double()
        nl = C.c_int64()
        self._c(_lib.hh_force_timing(self.h, int(enable), C.byref(ms), C.byref(nl)))
        return ms.value, nl.value


@dataclass
class Tree:
    """Output of the library's host tree builder (hh_tree_build)."""
    perm: np.ndarray
    node_x: np.ndarray  # [3, n_nodes]
    node_v: np.ndarray
    node_a: np.ndarray
    node_jk: np.ndarray
    node_m: np.ndarray
    off: np.ndarray
    idx: np.ndarray
    group_of: np.ndarray
    extra: dict = field(default_factory=dict)

    @property
    def n_nodes(self):
        return len(self.node_m)

    @property
    def n_groups(self):
        return len(self.off) - 1


def hh_tree_build(x, v, a, jk, m, leaf=8, n_crit=64, theta=0.5, order=0) -> Tree:
    """Host tree, groups and lists (SoA [3, n] inputs, any particle order);
    order HH_ORDER_MORTON (0) or HH_ORDER_HILBERT (1)."""
    n = len(m)
    arrs = [_f64(u, (3, n)) for u in (x, v, a, jk)] + [_f64(m, (n,))]
    h = _P()
    _check(_lib.hh_tree_build_ordered(C.byref(h), n, *[_ptr(u) for u in arrs], int(leaf), int(n_crit), float(theta),
                                      int(order)))
    try:
        nn, ng, ll = C.c_int64(), C.c_int32(), C.c_int64()
        _check(_lib.hh_tree_sizes(h, C.byref(nn), C.byref(ng), C.byref(ll)))
        nn, ng, ll = nn.value, ng.value, ll.value
        perm = np.zeros(n, np.int32)
        nx, nv, na, nj = (np.zeros((3, nn)) for _ in range(4))
        nm = np.zeros(nn)
        off = np.zeros(ng + 1, np.int64)
        idx = np.zeros(max(ll, 1), np.int32)
        gof = np.zeros(n, np.int32)
        _check(_lib.hh_tree_export(h, _ptr(perm, C.c_int32), _ptr(nx), _ptr(nv), _ptr(na), _ptr(nj), _ptr(nm),
                                   _ptr(off, C.c_int64), _ptr(idx, C.c_int32), _ptr(gof, C.c_int32)))
    finally:
        _lib.hh_tree_free(h)
    return Tree(perm, nx, nv, na, nj, nm, off, idx[:ll], gof)


_STATIC_DTYPES = {"xj": "float64", "vj": "float64", "mj": "float64", "off": "int64", "idx": "int32",
                  "i_idx": "int32", "gid": "int32", "acc": "float64", "jerk": "float64", "pot": "float64"}


def _static_check_args(device, **t):
    """Dtype, element count and device of every hh_force_static tensor, checked
    before the call: the C function trusts the pointers and sizes it gets, so a
    wrong dtype or a short buffer would make its kernels read or write past the
    caller's memory."""
    for name, u in t.items():
        if not hasattr(u, "numel") or not hasattr(u, "dtype"):
            raise ValueError(f"hh_force_static: {name} must be a tensor")
        want = _STATIC_DTYPES[name]
        if str(u.dtype).replace("torch.", "") != want:
            raise ValueError(f"hh_force_static: {name} must be {want}, got {u.dtype}")
        if not u.is_contiguous():
            raise ValueError(f"hh_force_static: {name} must be contiguous")
    n_j = t["mj"].numel()
    n_groups = t["off"].numel() - 1
    n_act = t["i_idx"].numel()
    sizes = {"xj": 3 * n_j, "vj": 3 * n_j, "gid": n_act, "acc": 3 * n_act, "jerk": 3 * n_act, "pot": n_act}
    for name, want in sizes.items():
        if t[name].numel() != want:
            raise ValueError(f"hh_force_static: {name} has {t[name].numel()} elements, expected {want}")
    if n_groups < 1:
        raise ValueError("hh_force_static: off needs at least two elements (n_groups >= 1)")
    for name, u in t.items():
        if not u.is_cuda or u.device.index != int(device):
            raise ValueError(f"hh_force_static: {name} must be on cuda:{int(device)}, got {u.device}")
    # the list length off[n_groups] must fit idx (one small device-to-host read)
    list_len = int(t["off"][-1].item())
    if list_len > t["idx"].numel():
        raise ValueError(f"hh_force_static: off[-1] = {list_len} exceeds idx's {t['idx'].numel()} elements")
    return n_j, n_groups, n_act


def hh_force_static(xj, vj, mj, off, idx, i_idx, gid, acc, jerk, pot, eps2=1e-8, precision=HH_FP64, device=0,
                    stream=None):
    """Allocation-free list force on caller-owned torch CUDA tensors (shapes
    and dtypes as in include/hh.h: float64 xj, vj [3, n_j], mj [n_j], acc,
    jerk [3, n_act], pot [n_act]; int64 off [n_groups + 1]; int32 idx,
    i_idx, gid).  Sizes are taken from mj, off and i_idx; every tensor is
    checked for dtype, element count and device before the call (ValueError).
    Raises HHError for the library's own errors."""
    n_j, n_groups, n_act = _static_check_args(device, xj=xj, vj=vj, mj=mj, off=off, idx=idx, i_idx=i_idx, gid=gid,
                                              acc=acc, jerk=jerk, pot=pot)
    s = stream if isinstance(stream, int) else (stream.cuda_stream if stream is not None else None)
    _check(_lib.hh_force_static(int(device), int(precision), float(eps2), n_j, _dev_ptr(xj), _dev_ptr(vj),
                                _dev_ptr(mj), n_groups, _dev_ptr(off), _dev_ptr(idx), n_act, _dev_ptr(i_idx),
                                _dev_ptr(gid), _dev_ptr(acc), _dev_ptr(jerk), _dev_ptr(pot), s))


class Batch:
    """Persistent batched block steps over many contexts (hh_batch_*)."""

    def __init__(self, precision=HH_FP64, max_sims=256, max_steps=4096, device=0):
        h = _P()
        _check(_lib.hh_batch_create(C.byref(h), int(device), int(precision), int(max_sims), int(max_steps)))
        self.h = h
        self.max_steps = int(max_steps)
        self.max_sims = int(max_sims)

    def close(self):
        if getattr(self, "h", None):
            _lib.hh_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def hh_batch_set_ctas(self, n_ctas):
        """CTAs (SMs) of the launches: > 0 that many, <= 0 all but |n_ctas|."""
        rc = _lib.hh_batch_set_ctas(self.h, int(n_ctas))
        if rc != HH_OK:
            raise HHError(rc, (_lib.hh_batch_last_error(self.h) or b"").decode())

    def hh_batch_run(self, ctxs, t_end, max_steps=None):
        """Runs the contexts until each passes its t_end (or max_steps global
        steps).  Returns (global steps, next block time per context, per-step
        durations in microseconds)."""
        n = len(ctxs)
        arr = (_P * n)(*[c.h for c in ctxs])
        te = np.ascontiguousarray(np.broadcast_to(np.asarray(t_end, dtype=np.float64), (n,)))
        ms = self.max_steps if max_steps is None else int(max_steps)
        steps = C.c_int32()
        tn = np.zeros(n)
        us = np.zeros(ms)
        ph = np.zeros((ms, 3))
        rc = _lib.hh_batch_run(self.h, n, arr, _ptr(te), ms, C.byref(steps), _ptr(tn), _ptr(us), _ptr(ph))
        if rc != HH_OK:
            raise HHError(rc, (_lib.hh_batch_last_error(self.h) or b"").decode())
        self.last_phase_us = ph[:steps.value]
        return steps.value, tn, us[:steps.value]

    def hh_batch_rebuild(self, ctxs, t, check=True):
        """Rebuilds the contexts at times t (device builders together, in one
        batched build).  Returns each context's status code; with check, a
        failure raises HHError."""
        n = len(ctxs)
        arr = (_P * n)(*[c.h for c in ctxs])
        tt = np.ascontiguousarray(np.broadcast_to(np.asarray(t, dtype=np.float64), (n,)))
        rcs = (C.c_int * n)()
        rc = _lib.hh_batch_rebuild(self.h, n, arr, _ptr(tt), rcs)
        if check and rc != HH_OK:
            raise HHError(rc, (_lib.hh_batch_last_error(self.h) or b"").decode())
        return [rcs[k] for k in range(n)]


    def _bcheck(self, rc):
        if rc != HH_OK:
            raise HHError(rc, (_lib.hh_batch_last_error(self.h) or b"").decode())

    # -- resident set (admission by budget, continuous batching) --------------
    def hh_batch_set_budget(self, budget_bytes=0, launch_particles=0):
        self._bcheck(_lib.hh_batch_set_budget(self.h, int(budget_bytes), int(launch_particles)))

    def hh_batch_admit(self, ctx, t_end):
        """Admits ctx to run to t_end; returns False (nothing changes) when no
        slot is free or its device bytes do not fit the budget."""
        rc = _lib.hh_batch_admit(self.h, ctx.h, float(t_end))
        if rc == HH_ENOMEM:
            return False
        self._bcheck(rc)
        return True

    def hh_batch_step(self, max_steps=None):
        """One launch over the running residents plus their due rebuilds.
        Returns (global steps, simulations launched, handles of the contexts
        that reached their end time, per-step microseconds)."""
        ms = self.max_steps if max_steps is None else int(max_steps)
        steps, launched, nd = C.c_int32(), C.c_int32(), C.c_int32()
        done = (_P * self.max_sims)()
        us = np.zeros(ms)
        ph = np.zeros((ms, 3))
        self._bcheck(_lib.hh_batch_step(self.h, ms, C.byref(steps), C.byref(launched), C.byref(nd), done, _ptr(us),
                                        _ptr(ph)))
        self.last_phase_us = ph[:steps.value]
        return steps.value, launched.value, [done[k] for k in range(nd.value)], us[:steps.value]

    def hh_batch_retire(self, ctx):
        self._bcheck(_lib.hh_batch_retire(self.h, ctx.h))

    def hh_batch_resident(self):
        """(resident contexts, running ones, device bytes held against the budget)."""
        n, r, b = C.c_int32(), C.c_int32(), C.c_int64()
        self._bcheck(_lib.hh_batch_resident(self.h, C.byref(n), C.byref(r), C.byref(b)))
        return n.value, r.value, b.value


def hh_selftest_aarseth(A, J, S, T, eta, device=0):
    """Device value of the timestep criterion for squared norms A, J, S, T."""
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (A, J, S, T)]
    n = len(arrs[0])
    out = np.zeros(n)
    _check(_lib.hh_selftest_aarseth(int(device), n, *[_ptr(x) for x in arrs], float(eta), _ptr(out)))
    return out


def hh_selftest_block_dt(want, dt_old, t_new, dt_min, dt_max, device=0):
    """Device block quantisation of the corrector for arrays want, dt_old, t_new."""
    arrs = [np.ascontiguousarray(x, dtype=np.float64) for x in (want, dt_old, t_new)]
    n = len(arrs[0])
    out = np.zeros(n)
    _check(_lib.hh_selftest_block_dt(int(device), n, *[_ptr(x) for x in arrs], float(dt_min), float(dt_max), _ptr(out)))
    return out


def hh_barrier_selftest(skip_cta=-1, device=0):
    """Returns (status code, seconds): HH_ETIMEOUT expected when skip_cta >= 0."""
    t = C.c_double()
    rc = _lib.hh_barrier_selftest(int(device), int(skip_cta), C.byref(t))
    return rc, t.value

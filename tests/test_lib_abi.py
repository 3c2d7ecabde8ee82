"""Host-side checks of libhh (no GPU): exports, host tree builder, argument errors.

The host tree builder is the library's own implementation of tree-loop step 1
(Section 2); it shares no code with the oracle, and both follow the same
written rules, so their Morton order, groups and lists must agree exactly.
"""
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


@pytest.fixture(scope="module")
def hh():
    import __graft_entry__
    __graft_entry__.build_library()
    import paper_1602_02832_gb300 as hh
    return hh


def _declared():
    names = set()
    for h in HEADERS:
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(hh\w*)\s*\(", src):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(hh):
    declared = _declared()
    assert "hh_force" in declared and "hh_tree_build" in declared
    missing = [n for n in sorted(declared) if not hasattr(hh.lib(), n)]
    assert not missing, missing
    # and the Python binding wraps every one of them
    assert not (declared - set(hh.EXPORTED)) - {"hh_batch"}, declared - set(hh.EXPORTED)


def test_config_default(hh):
    c = hh.hh_config_default()
    assert c.dt_min == 2.0 ** -30 and c.dt_max == 2.0 ** -6 and c.dt_tree == 2.0 ** -6
    assert c.theta == 0.5 and c.leaf == 8 and c.precision == hh.HH_FP64


def test_create_rejects_bad_config_without_touching_the_gpu(hh):
    c = hh.hh_config_default()
    c.dt_max = 0.3  # not a power of two
    with pytest.raises(hh.HHError) as e:
        hh.Context(c, 16, 32, 64, 4)
    assert e.value.code == hh.HH_EINVAL
    c = hh.hh_config_default()
    c.dt_max = 2.0 ** -3  # larger than dt_tree
    with pytest.raises(hh.HHError):
        hh.Context(c, 16, 32, 64, 4)


def _soa(a):
    return np.ascontiguousarray(np.asarray(a).T)


@pytest.mark.parametrize("order", ["morton", "hilbert"])
@pytest.mark.parametrize("n,theta,n_crit,salp", [(3000, 0.5, 64, False), (2500, 0.3, 16, True),
                                                 (4096, 0.75, 200, False), (777, 0.0, 32, True)])
def test_host_tree_matches_oracle_exactly(hh, orc, n, theta, n_crit, salp, order):
    x, v, m = (synth.plummer_salpeter if salp else synth.plummer)(n, 21)
    a, j, _ = orc.direct_force(x, v, m, 1e-6)
    T = orc.tree_build(x, v, a, j, m, leaf=8, n_crit=n_crit, theta=theta, order=order)
    P = hh.hh_tree_build(_soa(x), _soa(v), _soa(a), _soa(j), m, leaf=8, n_crit=n_crit, theta=theta,
                         order=hh.HH_ORDER_HILBERT if order == "hilbert" else hh.HH_ORDER_MORTON)
    assert np.array_equal(P.perm, T.perm)
    assert P.n_nodes == T.n_cells
    assert np.array_equal(P.off, T.list_off)
    assert np.array_equal(P.idx, T.list_idx)
    assert np.array_equal(P.group_of, T.group_of)
    np.testing.assert_allclose(P.node_x.T, T.node_x, rtol=0, atol=0)
    np.testing.assert_allclose(P.node_m, T.node_m, rtol=0, atol=0)
    np.testing.assert_allclose(P.node_jk.T, T.node_j, rtol=1e-15, atol=0)


def _degenerate_positions():
    rng = np.random.default_rng(0)
    grid = np.stack(np.meshgrid(*[np.arange(4.0)] * 3, indexing="ij"), -1).reshape(-1, 3)
    return {
        "one": np.array([[0.3, -0.2, 0.1]]),
        "two": np.array([[0.0, 0.0, 0.0], [1e-9, 0.0, 0.0]]),
        # all at one point: the depth limit (21) ends the split with one leaf
        "coincident": np.zeros((20, 3)),
        # a clump far below the finest cell of the root cube, and one outlier
        "clump_outlier": np.concatenate([rng.normal(size=(50, 3)) * 1e-7, [[1e3, 1e3, 1e3]]]),
        # ties on every cell boundary
        "grid": grid,
    }


@pytest.mark.parametrize("case", list(_degenerate_positions()))
@pytest.mark.parametrize("leaf,n_crit,theta", [(8, 4, 0.5), (1, 1, 0.75), (8, 64, 0.0)])
def test_host_tree_degenerate_inputs_match_oracle(hh, orc, case, leaf, n_crit, theta):
    x = _degenerate_positions()[case]
    n = len(x)
    rng = np.random.default_rng(1)
    v, a, j = (rng.normal(size=(n, 3)) for _ in range(3))
    m = rng.uniform(0.5, 1.5, n)
    T = orc.tree_build(x, v, a, j, m, leaf=leaf, n_crit=n_crit, theta=theta)
    P = hh.hh_tree_build(_soa(x), _soa(v), _soa(a), _soa(j), m, leaf=leaf, n_crit=n_crit, theta=theta)
    assert np.array_equal(P.perm, T.perm) and P.n_nodes == T.n_cells
    assert np.array_equal(P.off, T.list_off) and np.array_equal(P.idx, T.list_idx)
    assert np.array_equal(P.group_of, T.group_of)
    assert np.array_equal(P.node_m, T.node_m) and np.array_equal(P.node_x.T, T.node_x)


def test_host_tree_rejects_bad_inputs(hh):
    n = 20
    x = np.zeros((3, n))
    v = np.zeros((3, n))
    m = np.full(n, 1.0 / n)
    with pytest.raises(hh.HHError):
        hh.hh_tree_build(x, v, v, v, np.zeros(n))
    xx = x.copy()
    xx[0, 3] = np.nan
    with pytest.raises(hh.HHError):
        hh.hh_tree_build(xx, v, v, v, m)
    with pytest.raises(hh.HHError):
        hh.hh_tree_build(x, v, v, v, m, theta=-0.1)
    with pytest.raises(hh.HHError):
        hh.hh_tree_build(x, v, v, v, m, leaf=0)


def test_autotuner_candidates_are_valid_configurations(hh):
    # every candidate passes the library's configuration checks, which run
    # before any device call: on a machine without a GPU a valid candidate
    # gets past them (and fails only at the device), an invalid one is
    # refused with HH_EINVAL
    import torch
    from paper_1602_02832_gb300 import autotune

    if torch.cuda.is_available():
        pytest.skip("needs a machine without a GPU (no context is created)")
    for prec, cands in autotune.CANDIDATES.items():
        for cand in cands:
            c = hh.hh_config_default()
            c.precision = prec
            for k, v in cand.items():
                setattr(c, k, v)
            with pytest.raises(hh.HHError) as e:
                hh.Context(c, 16, 32, 64, 4)
            assert e.value.code != hh.HH_EINVAL, (prec, cand, str(e.value))
    c = hh.hh_config_default()
    c.precision = hh.HH_MIXED
    c.tile_j = 128  # not a multiple of the mixed form's 256-entry chunk
    with pytest.raises(hh.HHError) as e:
        hh.Context(c, 16, 32, 64, 4)
    assert e.value.code == hh.HH_EINVAL


@pytest.mark.parametrize("lang,std", [("c", "c99"), ("c++", "c++17")])
def test_header_is_plain_c_and_cpp(lang, std):
    # the boundary header compiles on its own as C99 and as C++ without warnings
    import shutil
    import subprocess

    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run([cc, f"-std={std}", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", lang,
                        os.path.join(inc, "hh.h")], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr


def test_binding_constants_match_header(hh):
    # every #define of the header has the same value in the binding, and every
    # error code has a name for HHError messages
    import re

    with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hh.h")) as f:
        hdr = f.read()
    defs = {k: int(v) for k, v in re.findall(r"#define (HH_[A-Z0-9_]+) \(?(-?\d+)\)?", hdr)}
    assert {"HH_OK", "HH_EINVAL", "HH_ESTATE", "HH_MIXED", "HH_ORDER_HILBERT"} <= set(defs)
    for k, v in defs.items():
        assert getattr(hh, k) == v, k
    for k, v in defs.items():
        if k.startswith("HH_E"):
            assert hh.HHError(v, "x").args[0].startswith(k + ":"), k


@pytest.mark.parametrize("sname", ["hh_config", "hh_counters"])
def test_binding_structs_match_header(hh, sname):
    # field names, order and sizes of the ctypes structures follow the header
    import ctypes as C
    import re

    with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hh.h")) as f:
        hdr = f.read()
    body = re.search(r"typedef struct %s \{(.*?)\} %s;" % (sname, sname), hdr, re.S).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    fields = re.findall(r"(double|int32_t|int64_t)\s+([a-z_0-9]+)\s*;", body)
    size = {"double": 8, "int32_t": 4, "int64_t": 8}
    cls = getattr(hh, sname)
    assert [n for n, _ in cls._fields_] == [n for _, n in fields]
    assert [C.sizeof(t) for _, t in cls._fields_] == [size[t] for t, _ in fields]
    assert all(t is not C.c_float for _, t in cls._fields_)
    assert [t in (C.c_double,) for _, t in cls._fields_] == [t == "double" for t, _ in fields]


def _kind_c(decl):
    decl = decl.strip()
    if "*" in decl or "[" in decl:
        return "ptr"
    base = decl.replace("const ", "").split()[0]
    return {"double": "f64", "int": "i32", "int32_t": "i32", "int64_t": "i64", "void": "void"}[base]


def _kind_ctypes(t):
    import ctypes as C

    if t is None:
        return "void"
    if t in (C.c_void_p, C.c_char_p) or hasattr(t, "_type_") and isinstance(t._type_, type):
        return "ptr"
    if t is C.c_double:
        return "f64"
    return {4: "i32", 8: "i64"}[C.sizeof(t)]


def test_binding_signatures_match_header(hh):
    # return and argument kinds (pointer, double, 32- or 64-bit integer) of
    # every bound call equal the header's prototype
    import re

    with open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "hh.h")) as f:
        hdr = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
    protos = {}
    for ret, name, args in re.findall(r"\n((?:const )?(?:int|void|int64_t|char)\s*\**)\s*(hh_\w+)\(([^)]*)\);", hdr):
        args = [a for a in (s.strip() for s in args.split(",")) if a and a != "void"]
        protos[name] = (_kind_c(ret), [_kind_c(a) for a in args])
    assert len(protos) >= 40
    sigs = hh._SIGS
    assert set(sigs) <= set(protos), set(sigs) - set(protos)
    for name, (res, args) in sigs.items():
        want_res, want_args = protos[name]
        assert _kind_ctypes(res) == want_res, name
        assert [_kind_ctypes(a) for a in args] == want_args, name


def test_force_static_binding_rejects_bad_tensors_before_any_call(hh, monkeypatch):
    # hh_force_static trusts its pointers and sizes, so the binding checks the
    # dtype, element count and device of every tensor first (ValueError).  The
    # C function is replaced by a recorder: none of these cases may reach it.
    torch = pytest.importorskip("torch")
    calls = []
    monkeypatch.setattr(hh, "_lib", _Recorder(hh._lib, calls))
    nj, na = 6, 2
    good = dict(xj=torch.zeros((3, nj), dtype=torch.float64), vj=torch.zeros((3, nj), dtype=torch.float64),
                mj=torch.ones(nj, dtype=torch.float64), off=torch.tensor([0, 3], dtype=torch.int64),
                idx=torch.tensor([0, 1, 2], dtype=torch.int32), i_idx=torch.tensor([0, 1], dtype=torch.int32),
                gid=torch.zeros(na, dtype=torch.int32), acc=torch.zeros((3, na), dtype=torch.float64),
                jerk=torch.zeros((3, na), dtype=torch.float64), pot=torch.zeros(na, dtype=torch.float64))
    bad_cases = [
        ("off", torch.tensor([0, 3], dtype=torch.int32), "int64"),
        ("idx", torch.tensor([0, 1, 2], dtype=torch.int64), "int32"),
        ("mj", torch.ones(nj, dtype=torch.float32), "float64"),
        ("gid", torch.zeros(na, dtype=torch.int64), "int32"),
        ("acc", torch.zeros((3, na + 1), dtype=torch.float64), "elements"),
        ("xj", torch.zeros((3, nj - 1), dtype=torch.float64), "elements"),
        ("pot", torch.zeros(na + 1, dtype=torch.float64), "elements"),
        ("jerk", torch.zeros((na, 3), dtype=torch.float64).t(), "contiguous"),
        ("xj", None, "tensor"),
    ]
    for name, val, word in bad_cases:
        args = dict(good, **{name: val})
        with pytest.raises(ValueError) as e:
            hh.hh_force_static(**args)
        assert word in str(e.value), (name, str(e.value))
    # well-typed host tensors are refused for their device
    with pytest.raises(ValueError) as e:
        hh.hh_force_static(**good)
    assert "cuda" in str(e.value)
    assert calls == []


class _Recorder:
    """Stands in for the loaded library: records hh_force_static calls, passes
    every other attribute through."""

    def __init__(self, lib, calls):
        self._lib, self._calls = lib, calls

    def hh_force_static(self, *a):
        self._calls.append(a)
        return 0

    def __getattr__(self, name):
        return getattr(self._lib, name)

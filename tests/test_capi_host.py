"""Host-side checks of the C ABI: the library builds for sm_103a, loads, exports every
entry point include/aexp.h declares, and rejects bad arguments before touching the GPU.
No call here launches device work."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2211_07532_gb300 import build
    build.build()
    import paper_2211_07532_gb300 as ax
    return ax.lib()


def declared_names():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^AEXP_API\s+(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", txt, re.M)
    return names


def test_every_declared_symbol_is_exported(L):
    names = declared_names()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_binding_covers_every_declared_symbol():
    import paper_2211_07532_gb300 as ax
    bound = {s[0] for s in ax.SIGNATURES}
    assert set(declared_names()) <= bound


def test_internal_symbols_are_hidden():
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2211_07532_gb300", "libaexp.so")],
                         capture_output=True, text=True).stdout
    assert "_ZN4aexp" not in out


def test_host_only_queries(L):
    import paper_2211_07532_gb300 as ax
    assert L.aexp_version() >= 100
    assert L.aexp_status_string(0) == b"ok"
    assert L.aexp_status_string(-8).startswith(b"workspace not prepared")
    o = ax.CReconOpts()
    L.aexp_recon_opts_default(ctypes.byref(o))
    assert (o.precision, o.wavelet, o.levels, o.n_power, o.use_graph) == (0, 0, 3, 30, 1)
    n = ctypes.c_size_t()
    assert L.aexp_wavelet_workspace_size(200, 200, 1, 4, ctypes.byref(n)) == 0
    assert n.value >= 208 * 208 * 8


def _fake_problem(nx=64, ny=64, nt=2048, nc=8, nl=9, omega=True):
    import paper_2211_07532_gb300 as ax
    base = 1 << 20  # fake, aligned, never dereferenced by host-only calls
    return ax.CProblem(nx, ny, nt, nc, nl, base, base + 4096, base if omega else None, base if omega else None, base)


def test_workspace_size_is_host_arithmetic(L):
    n = ctypes.c_size_t()
    p = _fake_problem()
    assert L.aexp_workspace_size(ctypes.byref(p), 0, ctypes.byref(n)) == 0
    # 8 coils -> 8 padded, 9 terms + B0 -> 12 padded; the reference phase table is one float per tile and sample
    assert n.value >= 64 * 2048 * 4
    p2 = _fake_problem(nx=200, ny=200, nt=24000, nc=32, nl=16)
    n2 = ctypes.c_size_t()
    assert L.aexp_workspace_size(ctypes.byref(p2), 0, ctypes.byref(n2)) == 0
    assert n2.value > n.value


def test_term_count_limit(L):
    """Up to 32 field terms with B0 (4th order = 25 harmonics, plus concomitant rows)."""
    n = ctypes.c_size_t()
    assert L.aexp_workspace_size(ctypes.byref(_fake_problem(nl=31)), 0, ctypes.byref(n)) == 0
    assert L.aexp_workspace_size(ctypes.byref(_fake_problem(nl=32, omega=False)), 0, ctypes.byref(n)) == 0
    assert L.aexp_workspace_size(ctypes.byref(_fake_problem(nl=32)), 0, ctypes.byref(n)) == -3


@pytest.mark.parametrize("field,value,code", [
    ("nx", 0, -1), ("nt", -3, -1), ("nc", 0, -1), ("nc", 33, -3), ("nl", 32, -3),
])
def test_invalid_problems_are_rejected(L, field, value, code):
    p = _fake_problem()
    setattr(p, field, value)
    n = ctypes.c_size_t()
    assert L.aexp_workspace_size(ctypes.byref(p), 0, ctypes.byref(n)) == code


def test_misaligned_and_null_pointers(L):
    import paper_2211_07532_gb300 as ax
    n = ctypes.c_size_t()
    p = _fake_problem()
    p.S = (1 << 20) + 4
    assert L.aexp_workspace_size(ctypes.byref(p), 0, ctypes.byref(n)) == -2
    p = _fake_problem()
    p.S = None
    assert L.aexp_workspace_size(ctypes.byref(p), 0, ctypes.byref(n)) == -1
    p = _fake_problem()
    # workspace checks happen before any launch
    assert L.aexp_prepare(ctypes.byref(p), 0, ctypes.c_void_p((1 << 30) + 8), 1 << 30, None) == -2
    assert L.aexp_prepare(ctypes.byref(p), 0, ctypes.c_void_p(1 << 30), 16, None) == -4
    assert L.a_exp_forward(ctypes.byref(p), 0, None, ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 30),
                           1 << 40, None) == -1
    # unprepared workspace
    assert L.a_exp_forward(ctypes.byref(p), 0, ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 20),
                           ctypes.c_void_p(1 << 30), 1 << 40, None) == -8
    # unsupported precision for now / bad enum
    assert L.aexp_workspace_size(ctypes.byref(p), 7, ctypes.byref(n)) == -1
    o = ax.CReconOpts()
    L.aexp_recon_opts_default(ctypes.byref(o))
    o.levels = 0
    assert L.aexp_recon_workspace_size(ctypes.byref(p), ctypes.byref(o), ctypes.byref(n)) == -1
    L.aexp_recon_opts_default(ctypes.byref(o))
    o.n_power = 0
    assert L.aexp_recon_workspace_size(ctypes.byref(p), ctypes.byref(o), ctypes.byref(n)) == -1
    o.lipschitz = 3.0
    assert L.aexp_recon_workspace_size(ctypes.byref(p), ctypes.byref(o), ctypes.byref(n)) == 0


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_2211_07532_gb300 as ax
    monkeypatch.setattr(ax, "_lib", None)
    monkeypatch.setattr(ax, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        ax.lib()


def test_items_per_sm_sizes_and_validation(L):
    """The work-item granularity changes only the partial-sum space; the tuner's workspace
    covers every candidate (granularity x tiling); out-of-range values are rejected on the host."""
    import paper_2211_07532_gb300 as ax
    p = _fake_problem(nx=200, ny=200, nt=24000, nc=32, nl=16)
    sizes = {}
    for prec in (ax.FP32, ax.BF16_TC, ax.FP16X2_TC):
        for ips in (0, 2, 4, 8, 16, 32):
            o = ax.CReconOpts()
            L.aexp_recon_opts_default(ctypes.byref(o))
            o.precision, o.items_per_sm = prec, ips
            n = ctypes.c_size_t()
            assert L.aexp_recon_workspace_size(ctypes.byref(p), ctypes.byref(o), ctypes.byref(n)) == 0
            sizes[(prec, ips)] = n.value
        # finer granularity -> more split partial sums -> never a smaller workspace
        assert sizes[(prec, 2)] <= sizes[(prec, 8)] <= sizes[(prec, 32)]
        # 0 is the default: 16 per SM for FP32, 8 for the tensor cores
        assert sizes[(prec, 0)] == sizes[(prec, 16 if prec == ax.FP32 else 8)]
        variants = (1,)   # 32 coils: every form has two tilings
        for v in variants:
            for ips in (2, 4, 8, 16, 32):
                o.items_per_sm, o.tile_variant = ips, v
                n = ctypes.c_size_t()
                assert L.aexp_recon_workspace_size(ctypes.byref(p), ctypes.byref(o), ctypes.byref(n)) == 0
                sizes[(prec, ips, v)] = n.value
        o.items_per_sm, o.tile_variant = 0, 0
        need = ctypes.c_size_t()
        assert L.aexp_autotune_workspace_size(ctypes.byref(p), 1, ctypes.byref(o), ctypes.byref(need)) == 0
        assert need.value == max([sizes[(prec, c)] for c in (2, 4, 8, 16, 32)] +
                                 [sizes[(prec, c, v)] for c in (2, 4, 8, 16, 32) for v in variants])
        # the operator-only workspace of a chosen launch shape; (0, 0) is aexp_workspace_size's
        w0, wt = ctypes.c_size_t(), ctypes.c_size_t()
        assert L.aexp_workspace_size(ctypes.byref(p), prec, ctypes.byref(w0)) == 0
        assert L.aexp_workspace_size_tiled(ctypes.byref(p), prec, 0, 0, ctypes.byref(wt)) == 0
        assert wt.value == w0.value
        for v in variants:
            assert L.aexp_workspace_size_tiled(ctypes.byref(p), prec, 8, v, ctypes.byref(wt)) == 0
        top = 2
        assert L.aexp_workspace_size_tiled(ctypes.byref(p), prec, 0, top, ctypes.byref(wt)) == -1
        assert L.aexp_workspace_size_tiled(ctypes.byref(p), prec, 257, 0, ctypes.byref(wt)) == -1
        assert L.aexp_prepare_tiled(ctypes.byref(p), prec, 0, top, None, 0, None) == -1
    for bad in (-1, 257):
        o.items_per_sm = bad
        assert L.aexp_recon_workspace_size(ctypes.byref(p), ctypes.byref(o), ctypes.byref(n)) == -1
    # the batched layout exists for the tensor-core precisions only
    o.items_per_sm = 0
    o.precision = ax.FP32
    arr = (ax.CProblem * 2)(p, _fake_problem(nx=148, ny=148, nt=8767, nc=32, nl=16))
    assert L.aexp_autotune_workspace_size(arr, 2, ctypes.byref(o), ctypes.byref(need)) == -3
    o.precision = ax.BF16_TC
    assert L.aexp_autotune_workspace_size(arr, 2, ctypes.byref(o), ctypes.byref(need)) == 0
    # no device call is made for a null workspace
    best = ctypes.c_int()
    variant = ctypes.c_int()
    assert L.aexp_autotune(arr, 2, ctypes.byref(o), None, 0, None, ctypes.byref(best), ctypes.byref(variant),
                           None) == -1
    o.tile_variant = 2   # out of range
    assert L.aexp_recon_workspace_size(ctypes.byref(p), ctypes.byref(o), ctypes.byref(n)) == -1
    o.tile_variant = 0

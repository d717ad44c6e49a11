"""C ABI checks that need no GPU: the library loads, exports every symbol
include/mg5.h declares, and its host-only entry points behave."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    return ctypes.CDLL(os.path.join(ROOT, "paper_1511_08200_gb300", "libmg5.so"))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(mg5_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_header_declares_the_boundary():
    d = _declared()
    for must in ("mg5_solve_fifth_force", "mg5_refine_interpolate", "mg5_relax_patch", "mg5_force",
                 "mg5_create", "mg5_destroy", "mg5_ndgp_coefficients"):
        assert must in d


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_entry_points(lib):
    lib.mg5_version.restype = ctypes.c_int
    assert lib.mg5_version() >= 100
    lib.mg5_status_string.restype = ctypes.c_char_p
    lib.mg5_status_string.argtypes = [ctypes.c_int]
    assert lib.mg5_status_string(0) == b"ok"
    assert b"invalid" in lib.mg5_status_string(-1)


def test_coefficients_match_oracle(lib):
    import oracle
    f = lib.mg5_ndgp_coefficients
    f.argtypes = [ctypes.c_double] * 3 + [ctypes.c_void_p] * 3
    f.restype = ctypes.c_int
    for a, om, rc in [(1.0, 0.3, 1.0), (0.5, 0.269, 1.0), (0.25, 0.3, 3.0)]:
        b, al, s = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        assert f(a, om, rc, ctypes.byref(b), ctypes.byref(al), ctypes.byref(s)) == 0
        ob, oal, os_ = oracle.ndgp_coefficients(a, om, rc)
        assert b.value == pytest.approx(ob, rel=1e-14)
        assert al.value == pytest.approx(oal, rel=1e-14)
        assert s.value == pytest.approx(os_, rel=1e-14)
    b = ctypes.c_double()
    assert f(0.0, 0.3, 1.0, ctypes.byref(b), None, None) == -1
    assert f(1.0, 1.5, 1.0, ctypes.byref(b), None, None) == -1


def test_workspace_bytes_and_size_rules(lib):
    f = lib.mg5_workspace_bytes
    f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    f.restype = ctypes.c_int
    out = ctypes.c_size_t()
    assert f(32, 0, ctypes.byref(out)) == 0
    # finest: tmp + f; coarse 16, 8, 4: v, tmp, f, v0
    assert out.value == 8 * (2 * 32 ** 3 + 4 * (16 ** 3 + 8 ** 3 + 4 ** 3))
    assert f(32, 1, ctypes.byref(out)) == 0 and out.value > 0
    assert f(31, 0, ctypes.byref(out)) == -1          # odd
    assert f(2, 0, ctypes.byref(out)) == -1           # too small
    assert f(2 * 33, 0, ctypes.byref(out)) == -1      # coarsest 66 > 32
    assert f(80, 0, ctypes.byref(out)) == 0           # 80 -> 40 -> 20 -> 10


def test_context_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib.mg5_create.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t]
    lib.mg5_create.restype = ctypes.c_int
    h = ctypes.c_void_p()
    rc = lib.mg5_create(ctypes.byref(h), 0, 0)
    assert rc in (-1, -3) and not h.value


def test_binding_imports_and_names(lib):
    import paper_1511_08200_gb300 as mg
    for name in ("solve_fifth_force", "refine_interpolate", "relax_patch", "force"):
        assert hasattr(mg.Context, name)
    p = mg.default_params(alpha=1.0, s=2.0, h=0.5)
    assert (p.nu1, p.nu2, p.tol, p.precision) == (2, 2, 1e-10, mg.FP64)
    assert mg.workspace_bytes(64, "mixed") > 0


def test_schedule_table_host_logic(lib, tmp_path):
    """The autotuner's table without a GPU: defaults, hand-set entries, validation,
    and the JSON-lines file round trip (entries for GPUs not present are skipped)."""
    import json
    import paper_1511_08200_gb300 as mg
    mg.tune_clear()
    s, tuned = mg.schedule_get(0, "fp64", 64)
    assert not tuned and (s.form, s.block) == (mg.SWEEP_TWO_PASS, 256)
    # 32^3 / 2 = 16384 threads: 16384 / 304 = 53 -> one warp a block, 512 blocks
    assert mg.schedule_get(0, "fp64", 32)[0].block == 32
    assert mg.schedule_get(0, "fp64", 48)[0].block == 160   # 55296 / 304 = 181 -> 160
    s, tuned = mg.schedule_get(0, "mixed", 64)
    assert not tuned and s.form == mg.SWEEP_MARCH          # a multiple of 32: the column march
    s, tuned = mg.schedule_get(0, "mixed", 48)
    assert not tuned and s.form == mg.SWEEP_FUSED          # fits the fused kernel only
    s, _ = mg.schedule_get(0, "mixed", 16)
    assert s.form == mg.SWEEP_TWO_PASS                     # below the fused kernel's minimum
    mg.schedule_set(0, "mixed", 64, mg.SWEEP_TWO_PASS, block=128)
    s, tuned = mg.schedule_get(0, "mixed", 64)
    assert tuned and (s.form, s.block) == (mg.SWEEP_TWO_PASS, 128)
    for bad in (dict(form=mg.SWEEP_TWO_PASS, block=33), dict(form=7), dict(form=1, chunk=-1)):
        with pytest.raises(mg.MG5Error):
            mg.schedule_set(0, "fp64", 32, **bad)
    path = tmp_path / "tune.jsonl"
    mg.schedule_set(0, "mixed", 96, mg.SWEEP_MARCH, chunk=24)
    mg.tune_save(path)
    rows = [json.loads(x) for x in path.read_text().splitlines()]
    assert rows == [{"gpu": rows[0]["gpu"], "precision": "mixed", "n": 64, "form": "two-pass",
                     "block": 128, "chunk": 0, "ms": 0},
                    {"gpu": rows[0]["gpu"], "precision": "mixed", "n": 96, "form": "march",
                     "block": 256, "chunk": 24, "ms": 0}]
    mg.tune_clear()
    assert not mg.schedule_get(0, "mixed", 64)[1]
    import torch
    if not torch.cuda.is_available():
        assert mg.tune_load(path) == 0                     # no GPU of that name here
    (tmp_path / "bad.jsonl").write_text("not a table\n")
    with pytest.raises(mg.MG5Error):
        mg.tune_load(tmp_path / "bad.jsonl")
    mg.tune_clear()


def test_masked_truncation_argument_checks(lib):
    """mg5_parent_force_mask and mg5_relax_patch_masked reject bad arguments before they touch
    the context or the device (the pointers below are never dereferenced)."""
    import paper_1511_08200_gb300 as mg
    I3 = ctypes.c_int * 3
    P = ctypes.c_void_p
    fm = lib.mg5_parent_force_mask
    fm.argtypes = [P, P, P, I3, ctypes.c_int, I3, I3, ctypes.c_double, P, P, P]
    fm.restype = ctypes.c_int
    ctx = ctypes.create_string_buffer(1 << 16)     # zero-filled stand-in, never read here
    buf = ctypes.create_string_buffer(64)
    c, g, m = ctypes.addressof(ctx), ctypes.addressof(buf), ctypes.addressof(buf)

    def call(pd, per, o, pn, theta, ctxp=c):
        return fm(ctxp, g, g, I3(*pd), per, I3(*o), I3(*pn), theta, m, None, None)

    E_ARG = -1
    assert call((8, 8, 8), 1, (0, 0, 0), (4, 4, 4), 0.1, ctxp=None) == E_ARG
    assert call((8, 8, 8), 1, (0, 0, 0), (4, 4, 4), -0.1) == E_ARG
    assert call((8, 8, 8), 1, (0, 0, 0), (4, 4, 4), float("nan")) == E_ARG
    assert call((8, 8, 8), 1, (0, 8, 0), (4, 4, 4), 0.1) == E_ARG        # o >= pd (periodic)
    assert call((8, 8, 8), 1, (0, 0, 0), (4, 9, 4), 0.1) == E_ARG        # pn > pd
    assert call((8, 8, 8), 0, (0, 6, 0), (4, 4, 4), 0.1) == E_ARG        # o + pn > pd (box)
    assert call((8, 0, 8), 1, (0, 0, 0), (4, 1, 4), 0.1) == E_ARG        # empty parent
    assert call((8, 8, 8), 1, (0, 0, 0), (4, 0, 4), 0.1) == E_ARG        # empty patch
    rm = lib.mg5_relax_patch_masked
    rm.argtypes = [P, P, I3, P, P, ctypes.c_double, P, P, P]
    rm.restype = ctypes.c_int
    prm = mg.default_params(alpha=1.0, s=1.0, h=0.5)
    pp = ctypes.addressof(prm)
    assert rm(c, g, I3(4, 4, 4), None, pp, 0.0, g, None, None) == E_ARG   # no mask
    assert rm(c, g, I3(4, 5, 4), m, pp, 0.0, g, None, None) == E_ARG      # odd side
    assert rm(c, g, I3(4, 4, 4), m, pp, float("inf"), g, None, None) == E_ARG
    bad = mg.default_params(alpha=1.0, s=1.0, h=0.5, omega=2.5)
    assert rm(c, g, I3(4, 4, 4), m, ctypes.addressof(bad), 0.0, g, None, None) == E_ARG


def test_every_entry_point_is_documented():
    """Each function include/mg5.h declares has a comment directly above it (or above the
    group of declarations it belongs to)."""
    txt = open(os.path.join(ROOT, "include", "mg5.h")).read().split("\n")
    decl = re.compile(r"^(?:int|long long|const char \*|double|size_t|void)\s+\*?(mg5_[a-z0-9_]+)\s*\(")
    undocumented = []
    for i, line in enumerate(txt):
        m = decl.match(line)
        if not m:
            continue
        j, found = i - 1, False
        while j >= 0:
            s = txt[j].strip()
            if s.endswith("*/") or s.startswith("/*") or s.startswith("*"):
                found = True
                break
            if s.endswith(");") or s.endswith(",") or decl.match(s) or s.startswith("const ") \
                    or s.startswith("double ") or s.startswith("mg5_"):
                j -= 1
                continue
            break
        if not found:
            undocumented.append(m.group(1))
    assert not undocumented, undocumented


def test_range_checked_build_compiles_and_loads(lib):
    """The -DMG5_BOUNDS variant builds (every kernel with its element accesses checked),
    exports the same boundary and says that it is the range-checked build; the ordinary
    build says it is not, and its check entry point reports nothing."""
    from paper_1511_08200_gb300 import _build
    path = _build.build(bounds=True)
    assert path.endswith("libmg5_bounds.so")
    blib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(blib, n)]
    assert not missing, missing
    assert blib.mg5_bounds_build() == 1
    assert lib.mg5_bounds_build() == 0
    buf = ctypes.create_string_buffer(64)
    lib.mg5_bounds_check.argtypes = [ctypes.c_char_p, ctypes.c_int]
    assert lib.mg5_bounds_check(buf, 64) == 0 and buf.value == b""
    lib.mg5_bounds_note.argtypes = [ctypes.c_void_p]
    assert lib.mg5_bounds_note(None) == 0

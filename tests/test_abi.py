"""The C ABI library: it builds, loads, exports every declared entry point, and its host-only
argument checks behave as documented. None of these tests needs a GPU."""
import os
import re

import numpy as np
import pytest

import paper_2006_10004_gb300 as tv

INF = float("inf")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(tvspec_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


def test_library_loads_and_exports_every_declared_symbol():
    lib = tv.load()
    names = _declared_functions()
    assert "tvspec_decompose" in names and "tvspec_submit" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # every binding signature refers to a declared function and vice versa
    assert set(tv._SIGS) == set(names)


def test_binding_signatures_have_the_declared_arity():
    text = open(os.path.join(ROOT, "include", "tvspec.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    for name, (_, argtypes) in tv._SIGS.items():
        m = re.search(r"\b" + name + r"\s*\(([^)]*)\)", text)
        assert m, name
        params = m.group(1).strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        assert len(argtypes) == n, (name, len(argtypes), n)


def test_status_strings_and_version():
    lib = tv.load()
    for code, name in tv.STATUS.items():
        assert lib.tvspec_status_str(code).decode() == name
    assert lib.tvspec_status_str(99).decode() == "TVSPEC_UNKNOWN"
    assert b"sm_103a" in lib.tvspec_version()


def test_config_layout_and_defaults_match_the_header():
    # tvspec_config_init writes every field of the C struct: run it on a Config followed by a
    # guard region; the binding's struct must end where the C one does (guard untouched, last
    # field written) and hold the documented defaults
    import ctypes

    n = ctypes.sizeof(tv.Config)
    buf = (ctypes.c_ubyte * (n + 64))(*([0xAB] * (n + 64)))
    tv.load().tvspec_config_init(ctypes.cast(buf, ctypes.POINTER(tv.Config)))
    assert bytes(buf[n:]) == b"\xab" * 64
    c = tv.Config.from_buffer(buf)
    want = dict(p_storage=0, warm_start=1, kernel=0, tile=-1, temporal_block=0, use_graphs=1,
                fast_math=1, mem_budget_bytes=0, max_batch=0, pdl=1, persistent=0,
                barrier_timeout_ms=2000, test_barrier_noshow=-1, resident=1, resident_variant=-1,
                acc_mode=0, tune_cache=None, test_fail_alloc=0, test_guard_bytes=0, tma=0)
    for k, v in want.items():
        assert getattr(c, k) == v, k
    assert abs(c.tau - 0.125) < 1e-9


def _header_fields(struct_name):
    """Member names of a typedef'd struct of include/tvspec.h, in declaration order."""
    text = open(os.path.join(ROOT, "include", "tvspec.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    m = re.search(r"typedef struct(?: \w+)? \{([^}]*)\} " + struct_name + ";", text)
    assert m, struct_name
    names = []
    for decl in m.group(1).split(";"):
        decl = decl.strip()
        if not decl:
            continue
        decl = re.sub(r"\[[^]]*\]", "", decl)  # array extents
        head, _, rest = decl.partition(",")
        names.append(re.findall(r"(\w+)\s*$", head)[0])
        names += [x.strip().lstrip("*").strip() for x in rest.split(",") if x.strip()]
    return names


@pytest.mark.parametrize("struct,binding", [("tvspec_config", "Config"), ("tvspec_request", "Request"),
                                            ("tvspec_stats", "Stats"), ("tvspec_crop", "Crop"),
                                            ("tvspec_training_request", "TrainingRequest"),
                                            ("tvspec_rof_request", "RofRequest")])
def test_binding_structs_follow_the_header(struct, binding):
    # same members in the same order as the C declarations (the binding passes these by pointer)
    fields = [n for n, _ in getattr(tv, binding)._fields_]
    renamed = {"lambda": "lam"}  # a Python keyword
    assert fields == [renamed.get(n, n) for n in _header_fields(struct)]


def test_tile_table():
    shapes = tv.tile_shapes()
    assert len(shapes) >= 8
    for s in shapes:
        assert s["V"] in (2, 4) and s["R"] * s["V"] <= 32 and 1 <= s["TB"] <= 16
        hx = (s["TB"] + s["V"] - 1) // s["V"] * s["V"]
        assert 32 * s["V"] - 2 * hx > 0 and s["RW"] * s["R"] - 2 * s["TB"] > 0
    assert tv.load().tvspec_tile_info(len(shapes), None, None, None, None) == tv.EINVAL


def test_validate_accepts_good_requests():
    assert tv.validate((64, 64), 0.5, 20, 200, (0, 2, 5, 10, INF)) == tv.OK
    assert tv.validate((1, 1), 1.0, 2, 0, (0, INF)) == tv.OK
    assert tv.validate((3, 700), 0.25, 60, 300, (0, 1, 2, 4, 8, 16, INF)) == tv.OK
    assert tv.validate((5, 5), 0.5, 4, 10, (0.5, 1.0, 3.0)) == tv.OK


@pytest.mark.parametrize("kw", [
    dict(f_shape=(0, 5)), dict(f_shape=(5, 0)), dict(K=1), dict(K=0), dict(dt=0.0), dict(dt=-1.0),
    dict(dt=float("nan")), dict(dt=INF), dict(n_inner=-1), dict(edges=(0.0,)),
    dict(edges=(0.0, 0.0, 1.0)), dict(edges=(0.0, 2.0, 1.0)), dict(edges=(-1.0, 1.0)),
    dict(edges=(0.0, INF, 5.0)), dict(edges=(0.0, float("nan"))), dict(edges=tuple(range(70))),
    dict(mem_kind=7),
])
def test_validate_rejects_bad_arguments(kw):
    args = dict(f_shape=(8, 8), dt=0.5, K=4, n_inner=10, edges=(0, 1, INF))
    args.update(kw)
    assert tv.validate(**args) == tv.EINVAL
    assert len(tv.load().tvspec_last_error()) > 0


def test_validate_rejects_non_finite_host_image():
    f = np.zeros((4, 4), np.float32)
    f[2, 3] = np.nan
    assert tv.validate((4, 4), 0.5, 4, 10, (0, INF), f=f) == tv.EINVAL
    f[2, 3] = np.inf
    assert tv.validate((4, 4), 0.5, 4, 10, (0, INF), f=f) == tv.EINVAL


def test_resident_variant_table():
    vs = tv.resident_variants()
    assert len(vs) >= 3
    assert {(v["max_H"], v["max_W"]) for v in vs} >= {(64, 64), (128, 64), (64, 128)}
    for v in vs:
        assert v["threads"] % 256 == 0 and v["threads"] <= 1024 and v["min_ctas_per_sm"] >= 1
    assert tv.load().tvspec_resident_variant_info(len(vs), None, None, None, None) == tv.EINVAL


def test_validate_filters():
    K = 6
    ok = [(np.ones(K - 1), 1.0), (np.linspace(0, 1, K - 1), 0.0)]
    assert tv.validate((8, 8), 0.5, K, 10, (0, INF), filters=ok) == tv.OK
    assert tv.validate((8, 8), 0.5, K, 10, (0, INF), filters=[(np.ones(K - 1), 1.0)] * 64) == tv.OK
    assert tv.validate((8, 8), 0.5, K, 10, (0, INF), filters=[(np.ones(K - 1), 1.0)] * 65) == tv.EINVAL
    h = np.ones(K - 1)
    h[2] = np.nan
    assert tv.validate((8, 8), 0.5, K, 10, (0, INF), filters=[(h, 1.0)]) == tv.EINVAL
    assert tv.validate((8, 8), 0.5, K, 10, (0, INF), filters=[(np.ones(K - 1), INF)]) == tv.EINVAL


def test_null_arguments_are_rejected_without_a_gpu():
    lib = tv.load()
    assert lib.tvspec_validate(None) == tv.EINVAL
    assert lib.tvspec_plan_create(None, 0, None) == tv.EINVAL
    assert lib.tvspec_decompose_ex(None, None, None) == tv.EINVAL
    assert lib.tvspec_decompose_batch(None, 0, None, None) == tv.EINVAL
    assert lib.tvspec_poll(None, 1) == tv.EINVAL
    assert lib.tvspec_plan_destroy(None) == tv.OK


def test_plan_create_without_gpu_reports_ecuda():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tv.TvSpecError) as ei:
        tv.Plan(0)
    assert ei.value.status == tv.ECUDA

"""CPU checks of the C ABI: the library loads and exports every function that
include/*.h declares; the host-side validation paths that need no GPU."""
import ctypes
import re
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]


def _declared_functions():
    names = set()
    for h in (ROOT / "include").glob("*.h"):
        text = h.read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:lc_status|const char\s*\*)\s+(lc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    path = __graft_entry__._build_module().build()
    return ctypes.CDLL(str(path))


def test_header_declares_api():
    names = _declared_functions()
    for required in ("lc_plan_workspace_size", "lc_plan_create", "lc_execute", "lc_adjoint", "lc_destroy",
                     "lc_plan_create_ragged", "lc_status_string"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_header():
    from paper_2411_00033_gb300 import binding
    assert set(_declared_functions()) <= set(binding.EXPORTED) | {"lc_status_string"}
    assert set(binding.EXPORTED) <= set(_declared_functions())


def test_workspace_size_and_validation():
    from paper_2411_00033_gb300 import binding as B
    assert B.lc_plan_workspace_size(1024, B.LC_L2C, 1, B.LC_F64) > 0
    # N = 1e6 plan: A-hat dominates (N_c * 324 doubles)
    big = B.lc_plan_workspace_size(1_000_000, B.LC_L2C, 1, B.LC_F64)
    assert 49107 * 324 * 8 < big < 49107 * 324 * 8 + 40_000_000
    for bad in [(0, 0, 1, 0), (10, 2, 1, 0), (10, 0, 0, 0), (10, 0, 1, 9)]:
        with pytest.raises(B.LegChebError) as e:
            B.lc_plan_workspace_size(*bad)
        assert e.value.status == 1
    opts = B.lc_plan_options_default()
    assert (opts.s_hat, opts.fixed_s, opts.slices) == (32, 0, 0)  # 0: slices chosen from n
    assert "INVALID" in B.lc_status_string(1)


def test_plan_create_rejects_small_workspace_without_touching_gpu():
    from paper_2411_00033_gb300 import binding as B
    with pytest.raises(B.LegChebError) as e:
        B.lc_plan_create(1024, B.LC_L2C, 1, B.LC_F64, 256, 16, 0)
    assert e.value.status == 2
    with pytest.raises(B.LegChebError) as e:
        B.lc_plan_create(1024, B.LC_L2C, 1, B.LC_F64, 0, 1 << 30, 0)
    assert e.value.status == 1
    with pytest.raises(B.LegChebError) as e:   # misaligned workspace
        B.lc_plan_create(1024, B.LC_L2C, 1, B.LC_F64, 1 << 20 | 8, 1 << 30, 0)
    assert e.value.status == 1


def test_null_plan_calls_fail_cleanly(lib):
    from paper_2411_00033_gb300 import binding as B
    B.load()
    with pytest.raises(B.LegChebError):
        B.lc_execute(None, 1, 2, 0, 1, 0, 1, 0)
    with pytest.raises(B.LegChebError):
        B.lc_destroy(None)


def test_static_limit_constant_matches_header():
    from paper_2411_00033_gb300 import binding as B
    text = (ROOT / "include" / "legcheb.h").read_text()
    m = re.search(r"#define\s+LC_STATIC_MAX_N\s+(\d+)", text)
    assert m and int(m.group(1)) == B.LC_STATIC_MAX_N


def test_static_entry_rejects_bad_arguments_without_gpu(lib):
    # validation happens before any CUDA call: these return LC_ERR_INVALID_ARG here
    f = lib.lc_direct_static
    f.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p]
    f.restype = ctypes.c_int
    a, b = ctypes.c_void_p(1 << 20), ctypes.c_void_p(1 << 21)
    from paper_2411_00033_gb300 import binding as B
    cases = [
        (0, B.LC_STATIC_MAX_N + 1, 1, a, b, 0, 1, 0, 1),  # above the static array
        (0, 0, 1, a, b, 0, 1, 0, 1),                      # n < 1
        (2, 10, 1, a, b, 0, 1, 0, 1),                     # bad direction
        (0, 10, 1, a, a, 0, 1, 0, 1),                     # aliased
        (0, 10, 1, a, b, 0, 1, 0, 0),                     # output element stride 0, n > 1
        (1, 10, 2, a, b, 10, 1, 0, 1),                    # output batch stride 0, batch > 1
        (0, 10, 1, a, b, 0, -1, 0, 1),                    # negative stride
    ]
    for c in cases:
        assert f(*c, None) == 1, c


def test_values_option_validation_without_gpu():
    # values at Chebyshev points: power-of-two n up to LC_VALUES_MAX_N, FP64 tiers, uniform plans
    from paper_2411_00033_gb300 import binding as B
    opts = B.lc_plan_options_default()
    assert opts.values == 0
    opts.values = 1
    assert B.lc_plan_workspace_size(512, B.LC_L2C, 3, B.LC_F64_SPLIT, opts) > \
        B.lc_plan_workspace_size(512, B.LC_L2C, 3, B.LC_F64_SPLIT)
    assert B.lc_plan_workspace_size(1000, B.LC_C2L, 2, B.LC_F64, opts) > 0  # any n: Bluestein
    for n, dt in ((B.LC_VALUES_MAX_N_ANY + 1, B.LC_F64), (B.LC_VALUES_MAX_N * 2, B.LC_F64), (1, B.LC_F64_DF),
                  (512, B.LC_F32)):
        with pytest.raises(B.LegChebError) as e:
            B.lc_plan_workspace_size(n, B.LC_C2L, 1, dt, opts)
        assert e.value.status == 5, (n, dt)
    with pytest.raises(B.LegChebError) as e:
        B.lc_plan_workspace_size_ragged([64, 128], B.LC_L2C, B.LC_F64_SPLIT, opts)
    assert e.value.status == 5
    opts.values = 2
    with pytest.raises(B.LegChebError) as e:
        B.lc_plan_workspace_size(512, B.LC_L2C, 1, B.LC_F64, opts)
    assert e.value.status == 1
    text = (ROOT / "include" / "legcheb.h").read_text()
    m = re.search(r"#define\s+LC_VALUES_MAX_N\s+(\d+)", text)
    assert m and int(m.group(1)) == B.LC_VALUES_MAX_N
    m = re.search(r"#define\s+LC_VALUES_MAX_N_ANY\s+(\d+)", text)
    assert m and int(m.group(1)) == B.LC_VALUES_MAX_N_ANY


def test_alpha_option_validation_without_gpu():
    # Gegenbauer parameter: 0 or 1/2 is Legendre; -1/2 < a <= LC_GEGENBAUER_MAX_ALPHA otherwise
    from paper_2411_00033_gb300 import binding as B
    opts = B.lc_plan_options_default()
    assert opts.alpha == 0.0
    base = B.lc_plan_workspace_size(5000, B.LC_C2L, 2, B.LC_F64_DF)
    for a in (0.5, 0.25, -0.49, 1.0, B.LC_GEGENBAUER_MAX_ALPHA):
        opts.alpha = a
        assert B.lc_plan_workspace_size(5000, B.LC_C2L, 2, B.LC_F64_DF, opts) == base
        assert B.lc_plan_workspace_size_ragged([64, 5000], B.LC_L2C, B.LC_F64_SPLIT, opts) > 0
    for a in (-0.5, -1.0, 2.0001, float("nan"), float("inf")):
        opts.alpha = a
        with pytest.raises(B.LegChebError) as e:
            B.lc_plan_workspace_size(5000, B.LC_L2C, 1, B.LC_F64, opts)
        assert e.value.status == 1, a
        with pytest.raises(B.LegChebError) as e:
            B.lc_plan_workspace_size_ragged([64, 5000], B.LC_L2C, B.LC_F64_SPLIT, opts)
        assert e.value.status == 1, a
    text = (ROOT / "include" / "legcheb.h").read_text()
    m = re.search(r"#define\s+LC_GEGENBAUER_MAX_ALPHA\s+([0-9.]+)", text)
    assert m and float(m.group(1)) == B.LC_GEGENBAUER_MAX_ALPHA


def test_set_band_validation_without_gpu():
    from paper_2411_00033_gb300 import binding as B
    lib = B.load()
    import ctypes
    assert lib.lc_plan_set_band(None, 0, 0) == 1
    # a plan handle is needed for the range checks; NULL is rejected before them
    text = (ROOT / "include" / "legcheb.h").read_text()
    assert "lc_status lc_plan_set_band(lc_plan plan, int32_t ctas, int32_t after_leaf);" in text


def test_split_schedule_validation_without_gpu():
    from paper_2411_00033_gb300 import binding as B
    lib = B.load()
    assert lib.lc_plan_set_split_schedule(None, 1) == 1
    assert lib.lc_plan_set_split_schedule(None, 0) == 1
    text = (ROOT / "include" / "legcheb.h").read_text()
    assert "lc_status lc_plan_set_split_schedule(lc_plan plan, int32_t persistent);" in text


def test_nodal_option_validation_without_gpu():
    # the nodal variant: LC_F64 and LC_F32, uniform plans
    from paper_2411_00033_gb300 import binding as B
    opts = B.lc_plan_options_default()
    assert opts.nodal == 0
    opts.nodal = 1
    for dt in (B.LC_F64, B.LC_F32):
        assert B.lc_plan_workspace_size(5000, B.LC_L2C, 2, dt, opts) > 0
    for dt in (B.LC_F64_DF, B.LC_F64_SPLIT):
        with pytest.raises(B.LegChebError) as e:
            B.lc_plan_workspace_size(5000, B.LC_L2C, 2, dt, opts)
        assert e.value.status == 5
    with pytest.raises(B.LegChebError) as e:
        B.lc_plan_workspace_size_ragged([64, 5000], B.LC_L2C, B.LC_F64_SPLIT, opts)
    assert e.value.status == 5
    opts.nodal = 2
    with pytest.raises(B.LegChebError) as e:
        B.lc_plan_workspace_size(5000, B.LC_L2C, 1, B.LC_F64, opts)
    assert e.value.status == 1

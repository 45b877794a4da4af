"""The C-ABI library builds, loads and exports every symbol that
include/stochq.h declares; host-only calls behave without a GPU."""

import ctypes
import os
import re

import pytest

from conftest import ROOT

HEADER = os.path.join(ROOT, "include", "stochq.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sq_[A-Za-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1405_4524_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["sq_create", "sq_destroy", "sq_load_gauge", "sq_build_clover", "sq_dslash_eo",
              "sq_solve", "sq_solve_batch", "sq_contract_pion", "sq_apply_M",
              "sq_pack_spinor", "sq_unpack_spinor", "sq_status_string", "sq_last_error"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol(lib):
    from paper_1405_4524_gb300 import stochq

    assert set(declared_functions()) == set(stochq.EXPORTS)
    for n in declared_functions():
        assert callable(getattr(stochq, n))


def test_host_only_calls(lib):
    from paper_1405_4524_gb300 import stochq

    assert stochq.sq_status_string(0) == "SQ_OK"
    assert "NOCONV" in stochq.sq_status_string(6)
    p = stochq.sq_default_params()
    assert p.inner_prec == stochq.SQ_F32 and p.max_iter > 0 and p.delta == 0.0
    # argument validation happens before any CUDA call
    for dims in [(4, 4, 4, 7), (4, 0, 4, 8), (3, 4, 4, 8)]:
        with pytest.raises(stochq.StochqError) as e:
            stochq.sq_create(dims)
        assert e.value.status == stochq.SQ_ERR_ARG
    with pytest.raises(stochq.StochqError) as e:
        stochq.sq_create((4, 4, 4, 8), t_bc=0)
    assert e.value.status == stochq.SQ_ERR_ARG


def test_default_params_chunk_and_inner_sums(lib):
    from paper_1405_4524_gb300 import stochq

    assert stochq.sq_default_params().chunk == 0  # 24 then 4 iterations per graph launch
    assert stochq.sq_inner_sum_bits() == 32


def test_sums64_variant_builds_and_is_selected_by_environment(lib, tmp_path):
    """The build variant with FP64 inner-iteration sums has its own objects
    and library, exports the same symbols, and STOCHQ_LIBRARY loads it."""
    import subprocess
    import sys

    from paper_1405_4524_gb300 import build

    path = build.build(variant="sums64")
    assert path == build.library_path("sums64") and path != build.library_path()
    var = ctypes.CDLL(path)
    assert not [n for n in declared_functions() if not hasattr(var, n)]
    code = "from paper_1405_4524_gb300 import stochq as s; print(s.LIBPATH, s.sq_inner_sum_bits())"
    env = dict(os.environ, STOCHQ_LIBRARY=path)
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         check=True).stdout.split()
    assert out == [path, "64"]
    with pytest.raises(ValueError):
        build.build(variant="no_such_variant")

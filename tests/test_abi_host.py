"""Host-side checks of the C ABI library (no GPU): it builds, loads, exports
every symbol include/priest.h declares, and its host Gaussian stream matches
the oracle's independent implementation bit for bit."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def priest():
    from paper_2309_08235_gb300 import build, priest as P

    build.build()
    return P


def declared_functions():
    src = open(os.path.join(ROOT, "include", "priest.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(priest_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_abi():
    names = declared_functions()
    for want in ("priest_create", "priest_destroy", "priest_project", "priest_plan", "priest_submit",
                 "priest_poll"):
        assert want in names


def test_library_exports_every_declared_symbol(priest):
    lib = priest.lib()
    names = declared_functions()
    assert sorted(priest.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n


def test_host_stream_matches_oracle(priest, oracle):
    for seed in list(range(0, 1001, 7)) + [2**63 + 5, 2**64 - 1]:
        for count in (1, 2, 33):
            a = priest.priest_rng_normal(seed, count)
            b = oracle.rng_normal(seed, count)
            assert np.array_equal(a, b), seed
    a = priest.priest_rng_normal(42, 100_003)
    b = oracle.rng_normal(42, 100_003)
    assert np.array_equal(a, b)


def test_rng_rejects_negative_count(priest):
    import ctypes as C

    assert priest.lib().priest_rng_normal(C.c_uint64(1), -1, None) == priest.PRIEST_ERR_INVALID


def test_create_validates_config_before_touching_the_gpu(priest):
    bad = priest.make_config(None, None, degree=3)
    with pytest.raises(priest.PriestError) as e:
        priest.priest_create(bad)
    assert e.value.status == priest.PRIEST_ERR_INVALID


def test_chol_selftest_validates_arguments_before_touching_the_gpu(priest):
    a = np.eye(4)
    for D, threads in ((0, 256), (49, 256), (4, 0), (4, 48), (4, 2048)):
        st = priest.lib().priest_chol_selftest(D, threads, a.ctypes.data_as(priest.C.c_void_p),
                                               a.ctypes.data_as(priest.C.c_void_p))
        assert st == priest.PRIEST_ERR_INVALID, (D, threads)

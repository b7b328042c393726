"""The C-ABI library loads and exports every entry point include/qsgw.h declares (no GPU needed)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "qsgw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qsgw_\w+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["qsgw_chi0_init", "qsgw_chi0_accumulate", "qsgw_chi0_finalize", "qsgw_eps_inv", "qsgw_chi0_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2506_03477_gb300 import native
    if not os.path.exists(native.LIB_PATH):
        from paper_2506_03477_gb300 import build
        build.build()
    lib = native.load()
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(native.EXPORTS) >= set(_declared())


def test_status_strings_without_gpu():
    from paper_2506_03477_gb300 import native
    assert native.qsgw_status_string(0) == "QSGW_OK"
    assert "DOMAIN" in native.qsgw_status_string(native.QSGW_ERR_DOMAIN)


def test_argument_errors_are_synchronous_without_gpu():
    from paper_2506_03477_gb300 import native
    with pytest.raises(native.QsgwError) as e:
        native.qsgw_chi0_init([], [0.1], 2.0, native.QSGW_FP64, stream=0)
    assert e.value.status == native.QSGW_ERR_ARG
    with pytest.raises(native.QsgwError) as e:
        native.qsgw_chi0_init([10], [0.1] * 17, 2.0, native.QSGW_FP64, stream=0)
    assert e.value.status == native.QSGW_ERR_ARG
    with pytest.raises(native.QsgwError) as e:  # the reserved TF32 form is rejected before any device work
        native.qsgw_chi0_init([10], [0.1], 2.0, native.QSGW_MIXED_TF32X3, stream=0)
    assert e.value.status == native.QSGW_ERR_ARG


def test_tile_plan_candidates_without_gpu():
    """The tuner's search space: the (up to) three widest tile widths with N = width * n_omega <= 256
    and a multiple of 16 that fit the kernel's shared memory, each with the default tail cut (0) and
    with none (1)."""
    from paper_2506_03477_gb300 import native
    assert native.qsgw_tile_plan_candidates(12) == [(20, 0), (20, 1), (16, 0), (16, 1), (12, 0), (12, 1)]
    for L in range(1, 17):
        c = native.qsgw_tile_plan_candidates(L)
        assert 2 <= len(c) <= 6 and all((t * L) % 16 == 0 and t * L <= 256 for t, _ in c)
        widths = [t for t, _ in c[::2]]
        assert widths == sorted(widths, reverse=True) and [p for _, p in c] == [0, 1] * len(widths)
    assert native.qsgw_tile_plan_candidates(0) == [] and native.qsgw_tile_plan_candidates(17) == []

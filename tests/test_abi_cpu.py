"""Host-side checks of the C ABI library: it loads, exports every declared
symbol, and its planners match the oracle's cluster tree and block cluster
trees (no GPU needed)."""
import os
import re

import numpy as np
import pytest

from oracle import admissibility, ordering

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1701_00182_gb300 import build as b

    b.build()
    import paper_1701_00182_gb300 as acr

    return acr.load_library()


def _declared():
    text = open(os.path.join(ROOT, "include", "acr.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(acr_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "acr_factor" in names and "acr_solve_transpose" in names
    for nm in names:
        assert hasattr(lib, nm), nm


def test_error_strings(lib):
    import paper_1701_00182_gb300 as acr

    msgs = {acr.acr_error_string(s) for s in range(7)}
    assert len(msgs) == 7
    assert "unknown" in acr.acr_error_string(99)


@pytest.mark.parametrize("n,leaf", [(8, 8), (16, 32), (64, 64), (128, 64), (32, 16)])
def test_planner_matches_oracle_tree(lib, n, leaf):
    import paper_1701_00182_gb300 as acr

    perm, ncut = acr.acr_plane_ordering(n, leaf)
    operm, levels = ordering.cluster_tree(n, leaf)
    np.testing.assert_array_equal(perm, np.array(operm, dtype=np.int32))
    assert list(ncut) == [len(nd[0]["cut"]) for nd in [lv for lv in levels[:-1]]]


@pytest.mark.parametrize("n,leaf", [(12, 8), (16, 24), (16, 512), (1, 4), (2048, 64)])
def test_planner_rejects_bad_sizes(lib, n, leaf):
    import paper_1701_00182_gb300 as acr

    with pytest.raises(acr.AcrError):
        acr.acr_plane_ordering(n, leaf)


def test_factor_rejects_bad_arguments_before_touching_the_device(lib):
    import paper_1701_00182_gb300 as acr

    with pytest.raises(acr.AcrError) as e:
        acr.acr_factor(12, None, 1e-6, 8)
    assert e.value.status == acr.ACR_ERR_ARG
    with pytest.raises(acr.AcrError) as e:
        acr.acr_factor(16, None, -1.0, 32)
    assert e.value.status == acr.ACR_ERR_ARG


@pytest.mark.parametrize("n,leaf", [(8, 4), (16, 16), (32, 64), (64, 64), (128, 64)])
@pytest.mark.parametrize("eta", [None, 0.5, 1.0, 2.0, 3.7])
def test_block_planner_matches_oracle_partition(lib, n, leaf, eta):
    """Section 2.1 block cluster tree (weak and standard admissibility):
    the planner's blocks equal the oracle's, entry for entry and in order."""
    import paper_1701_00182_gb300 as acr

    got = acr.acr_plan_blocks(n, leaf, eta)
    _, blocks = admissibility.block_partition(n, leaf, eta)
    ref = np.array([(l, t, s, 1 if lr else 0) for l, t, s, lr in blocks], dtype=np.int32)
    np.testing.assert_array_equal(got, ref)


def test_block_planner_rejects_bad_arguments(lib):
    import ctypes

    import paper_1701_00182_gb300 as acr

    with pytest.raises(acr.AcrError):
        acr.acr_plan_blocks(12, 8, 1.0)
    with pytest.raises(acr.AcrError):
        acr.acr_plan_blocks(16, 16, float("nan"))
    cnt = ctypes.c_long(0)
    buf = np.zeros(4 * 3, dtype=np.int32)
    st = lib.acr_plan_blocks(16, 16, 1.0, buf.ctypes.data, 3, ctypes.byref(cnt))
    assert st == acr.ACR_ERR_ARG and cnt.value > 3 and not buf.any()

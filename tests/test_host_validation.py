"""xpbd_create rejects invalid models before touching the GPU (runs on CPU)."""
import numpy as np
import pytest

from paper_2301_01396_gb300 import binding, build, scenes


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _status(sc):
    try:
        binding.Solver.from_scene(sc)
    except binding.XpbdError as e:
        return e.status
    return 0


def test_coloring_conflict_rejected():
    sc = scenes.plain_cloth(6)
    bad = sc.with_(color_offsets=np.array([0, sc.m], np.int32))
    assert _status(bad) == 2


def test_missing_and_duplicate_constraints_rejected():
    sc = scenes.plain_cloth(6)
    order = sc.color_order.copy()
    order[1] = order[0]
    assert _status(sc.with_(color_order=order)) == 2
    offs = sc.color_offsets.copy()
    offs[-1] -= 1
    assert _status(sc.with_(color_offsets=offs)) == 2


def test_index_out_of_range_rejected():
    sc = scenes.plain_cloth(6)
    d = sc.dist_idx.copy()
    d[3, 1] = sc.V
    assert _status(sc.with_(dist_idx=d)) == 1
    d[3, 1] = d[3, 0]
    assert _status(sc.with_(dist_idx=d)) == 1


def test_bad_masses_and_positions_rejected():
    sc = scenes.plain_cloth(6)
    w = sc.inv_mass.copy()
    w[2] = -1.0
    assert _status(sc.with_(inv_mass=w)) == 1
    x = sc.rest_x.copy()
    x[0, 0] = np.nan
    assert _status(sc.with_(rest_x=x)) == 1


def test_degenerate_rest_tet_rejected():
    sc = scenes.tet_block(2, steps=1)
    x = sc.rest_x.copy()
    t = sc.tet_idx[0]
    x[t[3]] = x[t[0]] + 0.5 * (x[t[1]] - x[t[0]])    # flat tet
    assert _status(sc.with_(rest_x=x)) == 1


def test_coupled_tet_coloring_rules():
    """With coupled tets the coloring lists the C_H ids only: the uncoupled coloring (which
    also lists C_D) and a C_D id in place of a C_H id are rejected."""
    from tests.helpers import small_tets
    sc = small_tets(2)
    assert _status(sc.with_(tet_coupled=True)) == 2
    cs = scenes.couple_tets(sc)
    order = cs.color_order.copy()
    order[0] = sc.n_tet + order[0]
    assert _status(cs.with_(color_order=order)) == 2


def test_membrane_model_rules():
    """A membrane triangle with zero rest area is rejected; so is a coloring that leaves a
    membrane out or lists an id past the membranes."""
    sc = scenes.membrane_cloth(4)
    uv = sc.memb_uv.copy()
    uv[3, 2] = uv[3, 0]
    assert _status(sc.with_(memb_uv=uv)) == 1
    offs = sc.color_offsets.copy()
    offs[-1] -= 1
    assert _status(sc.with_(color_offsets=offs)) == 2
    order = sc.color_order.copy()
    order[0] = sc.m + sc.n_memb
    assert _status(sc.with_(color_order=order)) == 2

"""Ensembles (members with different grids, stiffnesses and viscosities,
grouped into size classes, each kernel of a step one batched launch per
class) give the same states as the members stepped one by one, and match the
FP64 oracle."""
import numpy as np
import pytest

import oracle as O
import paper_1305_3976_gb300 as ib
from paper_1305_3976_gb300 import inputs as I

from test_gpu_step import assert_fp64, compare, make_pair, psi_bound, rel

pytestmark = pytest.mark.gpu


def _grid(sc, prec):
    g = ib.Grid(3, sc.n, rho=sc.rho, mu=sc.mu, dt=sc.dt, precision=prec, rotate_split=True)
    g.add_fiber(sc.X, sc.edges, sc.kappa, sc.rest, sc.tris)
    return g


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_ensemble_equals_members_stepped_alone(prec):
    members = I.ensemble_members(count=5, sizes=(16, 24, 32))
    ens_grids = [_grid(sc, prec) for sc in members]
    solo = [_grid(sc, prec) for sc in members]
    ens = ib.Ensemble(ens_grids)
    ens.step(1)
    ens.step(6)
    for g in solo:
        g.step(7)
    # atomics (and per-grid autotuned sweep shapes) reorder the FP32 sums; the psi
    # solve amplifies the difference in p by its conditioning
    tol = 1e-12 if prec == "fp64" else 1e-4
    for a, b in zip(ens_grids, solo):
        fa, fb = a.fields(), b.fields()
        for k in ("u", "v", "w", "p"):
            assert rel(fa[k], fb[k]) < tol, (k, rel(fa[k], fb[k]))
        assert np.max(np.abs(a.markers() - b.markers())) < (1e-13 if prec == "fp64" else 1e-7)
    # members can be stepped on their own afterwards
    ens_grids[0].step(1)
    ens.close()
    for g in ens_grids + solo:
        g.close()


def test_ensemble_member_matches_oracle():
    sc = I.ensemble_members(count=3, sizes=(16, 24))[1]
    ora, g = make_pair(sc, "fp64")
    other = _grid(I.ensemble_members(count=1, sizes=(32,), seed=7)[0], "fp64")
    ens = ib.Ensemble([other, g])
    ora.step(4)
    ens.step(4)
    e = compare(ora, g)
    assert_fp64(e, 4)
    assert e["psi"] < psi_bound(sc, 4), e
    ens.close()
    g.close()
    other.close()


def test_ensemble_more_members_than_one_launch_holds_and_mixed_precision():
    # 26 members of one size (seven groups of at most 4, each a batched
    # launch per kernel), two FP64 members of another size in their own
    # class, and one member without markers
    many = I.ensemble_members(count=26, sizes=(16,), seed=3)
    grids = [_grid(sc, "fp32") for sc in many]
    solo = [_grid(sc, "fp32") for sc in many]
    extra = I.ensemble_members(count=2, sizes=(24,), seed=4)
    g64 = [_grid(sc, "fp64") for sc in extra]
    s64 = [_grid(sc, "fp64") for sc in extra]
    bare = ib.Grid(3, 16, rho=1.0, mu=0.05, dt=5e-4, precision="fp32", rotate_split=True)
    bare.set_velocity(I.random_velocity(3, (16, 16, 16), seed=9, amplitude=0.1).astype(np.float32))
    bare_solo = ib.Grid(3, 16, rho=1.0, mu=0.05, dt=5e-4, precision="fp32", rotate_split=True)
    bare_solo.set_velocity(I.random_velocity(3, (16, 16, 16), seed=9, amplitude=0.1).astype(np.float32))
    ens = ib.Ensemble(grids + g64 + [bare])
    ens.step(5)
    for g in solo + s64 + [bare_solo]:
        g.step(5)
    for a, b in zip(grids + [bare], solo + [bare_solo]):
        assert rel(a.velocity(), b.velocity()) < 1e-5
    for a, b in zip(g64, s64):
        assert rel(a.velocity(), b.velocity()) < 1e-12
        assert np.max(np.abs(a.markers() - b.markers())) < 1e-13
    ens.close()
    for g in grids + solo + g64 + s64 + [bare, bare_solo]:
        g.close()


def test_ensemble_rejects_mismatched_members():
    a = ib.Grid(3, 16, precision="fp32")
    b = ib.Grid(2, 16, precision="fp32")
    with pytest.raises(ib.IBError) as ex:
        ib.Ensemble([a, b])
    assert ex.value.code == ib.IB_ERR_STATE
    a.close()
    b.close()

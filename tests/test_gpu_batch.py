"""GPU parity of the ensemble path (lat_batch_*): members of uneven size and
coupling stepped by one persistent launch, against the FP64 oracle member by
member (FP32 2e-6 per step, FP64 1e-12 per step, normwise), against the
single-lattice path, and the bounded grid barrier's timeout."""
import numpy as np
import pytest

from gpu_helpers import normwise
from oracle.oracle import Oracle
from paper_0911_5692_gb300 import Ensemble, Lattice
from paper_0911_5692_gb300.workloads import ensemble_64, lphi4, m2phi2, random_state

pytestmark = pytest.mark.gpu

TOL = {32: 2e-6, 64: 1e-12}


def _members(prec, sizes=(32, 48, 64, 96, 32, 48), expansion=1):
    ps, states = [], []
    for i, n in enumerate(sizes):
        if i % 3 == 2:
            p = m2phi2(n, precision=prec, expansion=expansion, seed=i)
            st = random_state(n, 10 + i, prec, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-4), pi_mean=(0.3, 0.0),
                              pi_amp=(1e-3, 1e-2))
        else:
            p = lphi4(n, precision=prec, G=50.0 * (i + 1), expansion=expansion, seed=i)
            st = random_state(n, 10 + i, prec, f_mean=(1.0, 0.0), f_amp=(1e-3, 1e-3), pi_mean=(0.5, 0.0),
                              pi_amp=(1e-3, 1e-3))
        ps.append(p)
        states.append(st)
    return ps, states


SCAL = dict(t=0.0, a=1.05, ad=0.4, step=0)


def _load(ens, states, scal=SCAL):
    for i, st in enumerate(states):
        ens.member(i).set_state(*st, **scal)


@pytest.mark.parametrize("prec", [32, 64])
def test_members_match_oracle(prec):
    ps, states = _members(prec)
    ens = Ensemble(ps)
    _load(ens, states)
    steps = 6
    ens.evolve(steps)
    ens.sync()
    info = ens.info()
    assert info["launches"] == 1 and info["members"] == len(ps)
    for i, (p, st) in enumerate(zip(ps, states)):
        o = Oracle(p)
        o.set_state(*st, **SCAL)
        o.step(steps)
        m = ens.member(i)
        for a, b in zip(m.get_state(), o.get_state()):
            assert normwise(a, b) <= steps * TOL[prec], (i, normwise(a, b))
        gs, os_ = m.scalars(), o.scalars()
        assert gs["step"] == steps
        assert abs(gs["a"] / os_["a"] - 1) <= (1e-13 if prec == 64 else 1e-7)


def test_matches_single_lattice_path_fp64():
    ps, states = _members(64, sizes=(32, 64, 96))
    ens = Ensemble(ps)
    _load(ens, states)
    ens.evolve(9)
    for i, (p, st) in enumerate(zip(ps, states)):
        g = Lattice(p)
        g.set_state(*st, **SCAL)
        g.evolve(9)
        for a, b in zip(ens.member(i).get_state(), g.get_state()):
            assert normwise(a, b) <= 1e-13


def test_split_calls_are_bit_identical():
    ps, states = _members(32)
    a = Ensemble(ps)
    b = Ensemble(ps)
    _load(a, states)
    _load(b, states)
    a.evolve(7)
    b.evolve(3)
    b.evolve(4)
    for i in range(len(ps)):
        for x, y in zip(a.member(i).get_state(), b.member(i).get_state()):
            assert np.array_equal(x, y)
        assert a.member(i).scalars() == b.member(i).scalars()


def test_tune_restores_state_and_keeps_results():
    ps, states = _members(32)
    ens = Ensemble(ps)
    _load(ens, states)
    before = [ens.member(i).get_state() for i in range(len(ps))]
    ens.tune(3)
    for i in range(len(ps)):
        for x, y in zip(ens.member(i).get_state(), before[i]):
            assert np.array_equal(x, y)
    ens.evolve(4)
    ens.sync()
    for i, (p, st) in enumerate(zip(ps, states)):
        o = Oracle(p)
        o.set_state(*st, **SCAL)
        o.step(4)
        for a, b in zip(ens.member(i).get_state(), o.get_state()):
            assert normwise(a, b) <= 4 * TOL[32]


def test_tuned_shape_is_taken_by_new_ensembles():
    """lat_batch_tune sweeps block size x tile-height cap x prefetch depth; every
    member's tile height divides its side and stays within 32, and an ensemble
    created later with the same sizes and precision starts with the tuned shape."""
    ps, states = _members(32, sizes=(32, 64, 96))
    ens = Ensemble(ps)
    _load(ens, states)
    ens.tune(3)
    info = ens.info()
    assert len(info["ty"]) == len(ps)
    assert info["depth"] in (1, 2)
    for p, ty in zip(ps, info["ty"]):
        assert 1 <= ty <= 32 and p["n"] % ty == 0
    again = Ensemble([dict(p, seed=p["seed"] + 100) for p in ps])
    info2 = again.info()
    assert (info2["threads"], info2["ty"], info2["depth"]) == (info["threads"], info["ty"], info["depth"])
    _load(again, states)
    again.evolve(3)
    again.sync()
    for i, (p, st) in enumerate(zip(ps, states)):
        o = Oracle(p)
        o.set_state(*st, **SCAL)
        o.step(3)
        for a, b in zip(again.member(i).get_state(), o.get_state()):
            assert normwise(a, b) <= 3 * TOL[32]


@pytest.mark.parametrize("prec", [32, 64])
@pytest.mark.parametrize("threads,cap,depth", [(192, 4, 2), (256, 8, 2), (512, 32, 2), (384, 16, 1)])
def test_launch_shapes_match_oracle(prec, threads, cap, depth):
    """Every shape the tuner may pick steps the members as the oracle does: one
    or two planes in flight, tile heights from 4 to 32 (many short ranges per
    member at the small caps)."""
    ps, states = _members(prec)
    ens = Ensemble(ps)
    _load(ens, states)
    ens.set_shape(threads, cap, depth)
    info = ens.info()
    assert (info["threads"], info["tile_cap"], info["depth"]) == (threads, cap, depth)
    steps = 5
    ens.evolve(steps)
    ens.sync()
    for i, (p, st) in enumerate(zip(ps, states)):
        o = Oracle(p)
        o.set_state(*st, **SCAL)
        o.step(steps)
        for a, b in zip(ens.member(i).get_state(), o.get_state()):
            assert normwise(a, b) <= steps * TOL[prec], (i, normwise(a, b))


def test_set_shape_refusals():
    """Out-of-range shapes are LAT_EINVAL; a block too small for a member's
    tile is LAT_EUNSUPPORTED; the ensemble keeps its shape and still steps."""
    from paper_0911_5692_gb300.lattice import LatticeError
    ps, states = _members(32, sizes=(32, 96))
    ens = Ensemble(ps)
    _load(ens, states)
    before = ens.info()
    for args in ((256, 8, 3), (256, 0, 1), (16, 8, 1), (2048, 8, 1)):
        with pytest.raises(LatticeError) as e:
            ens.set_shape(*args)
        assert e.value.status == 1
    with pytest.raises(LatticeError) as e:
        ens.set_shape(64, 32, 1)          # a side-96 tile needs (ty + 3) rows of 24 threads: none fits 64
    assert e.value.status == 7
    after = ens.info()
    assert (after["threads"], after["ty"], after["depth"]) == (before["threads"], before["ty"], before["depth"])
    ens.evolve(2)
    ens.sync()


def test_static_members():
    ps, states = _members(64, sizes=(32, 48), expansion=0)
    ens = Ensemble(ps)
    _load(ens, states, dict(t=0.0, a=1.0, ad=0.0, step=0))
    ens.evolve(5)
    for i, (p, st) in enumerate(zip(ps, states)):
        o = Oracle(p)
        o.set_state(*st, t=0.0, a=1.0, ad=0.0, step=0)
        o.step(5)
        for a, b in zip(ens.member(i).get_state(), o.get_state()):
            assert normwise(a, b) <= 5 * TOL[64]


def test_barrier_wait_is_bounded():
    """A barrier that can never complete ends every block's wait after the
    timeout; the call reports LAT_ETIMEOUT and the context stays usable."""
    ps, states = _members(32, sizes=(32, 48))
    ens = Ensemble(ps)
    _load(ens, states)
    assert ens.check_barrier(200_000_000) == 6
    ens.evolve(2)
    ens.sync()
    o = Oracle(ps[0])
    o.set_state(*states[0], **SCAL)
    o.step(2)
    for a, b in zip(ens.member(0).get_state(), o.get_state()):
        assert normwise(a, b) <= 2 * TOL[32]


def test_full_ensemble_one_step_parity():
    """The 64-member ensemble (N in 32, 48, 64, 96; g^2/lambda log-uniform in
    [50, 500]) after initialisation: one step of sampled members against the
    oracle from the same stored state."""
    ps = ensemble_64()
    ens = Ensemble(ps)
    ens.init_fields()
    ens.evolve(3)
    ens.sync()
    picks = [0, 1, 2, 3, 37, 63]
    before = {i: (ens.member(i).get_state(), ens.member(i).scalars()) for i in picks}
    ens.evolve(1)
    ens.sync()
    for i in picks:
        st, sc = before[i]
        o = Oracle(ps[i])
        o.set_state(*st, t=sc["t"], a=sc["a"], ad=sc["ad"], step=sc["step"])
        o.step(1)
        for a, b in zip(ens.member(i).get_state(), o.get_state()):
            assert normwise(a, b) <= TOL[32], (i, normwise(a, b))

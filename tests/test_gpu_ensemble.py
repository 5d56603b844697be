"""Ensembles of uneven boxes in batched launches (one launch per sweep for all
boxes, per-box CFL timestep, CUDA-graph replay) against single boxes and the
FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1004_1680_gb300 import initial_conditions as ic
from tests.parity_util import G, field_scales, from_gpu, rel_err

pytestmark = pytest.mark.gpu

DIMS = [(32, 48, 32), (48, 32, 64), (64, 64, 32), (32, 32, 96), (96, 48, 32)]


@pytest.fixture(scope="module")
def mhd():
    from paper_1004_1680_gb300 import mhd as m
    m.load()
    return m


def states():
    out = []
    for b, d in enumerate(DIMS):
        st = ic.turbulence(d, seed=1000 + b, mach=0.5 + 0.3 * b, beta=0.3 + 0.6 * b,
                           dtype=torch.float64, kmin=1.0, kmax=4.0)
        out.append(st)
    return out


def make_ens(mhd, sts, xpath=2, segdiv=1):
    ens = mhd.Ensemble(DIMS, gamma=G)
    ens.set_tuning(xpath, segdiv)
    for b, st in enumerate(sts):
        ens.set_state(b, st.to(torch.float32).contiguous().cuda())
    return ens


@pytest.mark.parametrize("xpath,segdiv", [(2, 1), (1, 2)])
def test_members_equal_single_boxes(mhd, xpath, segdiv):
    sts = states()
    ens = make_ens(mhd, sts, xpath, segdiv)
    ens.run(3, 0.7)
    t = ens.times()
    for b, st in enumerate(sts):
        box = mhd.Box(*DIMS[b], gamma=G)
        box.set_xpath(xpath)
        box.set_tma(False)  # the ensemble's register-load sweeps
        box.set_state(st.to(torch.float32).contiguous().cuda())
        box.run(3, 0.7)
        assert torch.equal(ens.get_state(b), box.get_state()), b
        assert t[b] == box.time()
        assert np.array_equal(ens.diagnostics()[b], box.diagnostics())
        box.close()


def test_sampled_members_against_oracle(mhd):
    sts = states()
    ens = make_ens(mhd, sts)
    ens.run(4, 0.7)
    t = ens.times()
    for b in (0, 2, 3, 4):
        s = ic.as_oracle_input(sts[b])
        S = field_scales(s)
        t_orc, _ = oracle.run(s, 4, 0.7, G)
        assert t[b] == pytest.approx(t_orc, rel=1e-5)
        err = rel_err(from_gpu(ens.get_state(b)), s, S)
        assert np.all(err < 1e-4), (b, err)


def test_graph_replay_and_run_lengths(mhd):
    sts = states()
    a = make_ens(mhd, sts)
    a.run(2, 0.7)
    a.run(2, 0.7)          # second replay of the same cached graph
    a.run(3, 0.7)          # a different run length (new graph)
    b = make_ens(mhd, sts)
    b.run(7, 0.7)
    for k in range(len(DIMS)):
        assert torch.equal(a.get_state(k), b.get_state(k)), k
    assert np.array_equal(a.times(), b.times())


def test_autotune_keeps_state(mhd):
    sts = states()
    a = make_ens(mhd, sts)
    before = [a.get_state(k).clone() for k in range(len(DIMS))]
    xp, sd = a.autotune(0.7)
    assert xp in (1, 2) and sd in (1, 2)
    for k in range(len(DIMS)):
        assert torch.equal(a.get_state(k), before[k])
    assert np.all(a.times() == 0.0)
    a.run(2, 0.7)
    b = make_ens(mhd, sts, xp, sd)
    b.run(2, 0.7)
    for k in range(len(DIMS)):
        assert torch.equal(a.get_state(k), b.get_state(k))


def test_per_box_cfl_dt(mhd):
    sts = states()
    ens = make_ens(mhd, sts)
    dts = ens.cfl_dt(0.7)
    for b, st in enumerate(sts):
        assert dts[b] == pytest.approx(oracle.cfl_dt(ic.as_oracle_input(st), G, 0.7), rel=2e-6)

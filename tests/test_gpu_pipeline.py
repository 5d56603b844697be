"""Pipelined host runs (mhd_submit / mhd_drain): every submission's result
equals, bitwise, the same run done with set_state / run / get_state, with
several submissions in flight through the three rotating staging copies, on
both x paths; other calls are ordered after the submitted copies."""
import pytest
import torch

from paper_1004_1680_gb300 import initial_conditions as ic

pytestmark = pytest.mark.gpu
G = 5.0 / 3.0


@pytest.fixture(scope="module")
def mhd():
    from paper_1004_1680_gb300 import mhd as m
    m.load()
    return m


def states(n, k):
    return [ic.turbulence(n, seed=30 + i, dtype=torch.float64, kmin=1.0, kmax=3.0).to(torch.float32)
            .contiguous().pin_memory() for i in range(k)]


@pytest.mark.parametrize("xpath", [1, 2])
def test_submissions_equal_synchronous_runs(mhd, xpath):
    n = (32, 24, 20)
    ins = states(n, 5)
    ref = []
    box = mhd.Box(*n, gamma=G)
    box.set_xpath(xpath)
    for s in ins:
        box.set_state(s)
        box.run(2, 0.7)
        ref.append(box.get_state(device="cpu"))
    outs = [torch.empty_like(s).pin_memory() for s in ins]
    for s, o in zip(ins, outs):          # 5 in flight: every staging slot reused
        box.submit(s, o, 2, 0.7)
    box.drain()
    for i, (o, r) in enumerate(zip(outs, ref)):
        assert torch.equal(o, r), i
    # the box holds the last result; later calls are ordered after the copies
    assert torch.equal(box.get_state(device="cpu"), ref[-1])
    box.set_state(ins[0])
    box.run(2, 0.7)
    assert torch.equal(box.get_state(device="cpu"), ref[0])
    box.close()


def test_other_calls_wait_for_submitted_copies(mhd):
    n = (32, 24, 20)
    ins = states(n, 2)
    box = mhd.Box(*n, gamma=G)
    out0 = torch.empty_like(ins[0]).pin_memory()
    out1 = torch.empty_like(ins[1]).pin_memory()
    box.submit(ins[0], out0, 1, 0.7)
    box.submit(ins[1], out1, 1, 0.7)
    last = box.get_state(device="cpu")   # no drain: ordered after submission 1
    box.drain()
    assert torch.equal(last, out1)
    box.close()

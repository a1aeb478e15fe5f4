"""The one-launch step schedule (lbpf_set_schedule) on the GPU.

The one-launch kernel runs the same tile code as the two-kernel step, only ordered by
tickets and done flags, so every field must agree bit for bit with the two-kernel step
(which the parity tests pin to the oracle) for every storage type and instantiated lattice
triple, under tilings whose U/theta rings reach one or two z-chunks away, in single steps
and in graph replays, for single handles and for batches.  The bounded wait that the
launch's blocks use is exercised on its own: it returns when the flag is set, gives up on
a flag that nothing sets, and the device stays usable after it gave up; and a step whose
waits are bounded to nothing reports LBPF_ETIMEOUT on its handle.
"""
import time

import numpy as np
import pytest

from paper_1602_07483_gb300 import build, lbpf, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build.build()
    lbpf.load()


CASES = {
    # lattice triple (19, 19, 19): the 512^3 two-harmonic workload's recipe on a small box
    "q19x3": lambda: workloads.large_kh(n=70),
    # (19, 19, 7): coupled heat and solute
    "q19q19q7": lambda: workloads.coupled_dendrite(n=44),
    # (19, 19, 0): theta frozen, a member of the batched sweep
    "q19q19q0": lambda: workloads.batch_sweep(count=1)[0],
    # (9, 5, 5): the 2D benchmark of Sec. 4.1 on one-row blocks
    "d2q9": lambda: workloads.pure_substance_2d(n=130),
}


def _same(a, b):
    for x, y in zip(a.read_fields(), b.read_fields()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("case", sorted(CASES))
def test_one_launch_matches_two_kernels_bitwise(case, storage):
    w = CASES[case]()
    a = lbpf.sim_from_workload(w, storage=storage)
    b = lbpf.sim_from_workload(w, storage=storage)
    b.set_schedule("one_launch")
    assert a.schedule == "two_kernels" and b.schedule == "one_launch"
    for n in (1, 4, 13):  # single launches, then graph replays from a count that is not a multiple of 6
        a.step(n)
        b.step(n)
    assert b.steps_done == 18
    _same(a, b)
    assert np.array_equal(a.sums(), b.sums())


@pytest.mark.parametrize("tiling", [(4, 1), (5, 2), (8, 7)])
def test_one_launch_small_chunks_bitwise(tiling):
    """z-chunks of one and two planes: the U/theta ring then reads phi^{n+1} written by
    tiles two chunks away, which must all be waited for."""
    w = workloads.coupled_dendrite(n=40)
    a = lbpf.sim_from_workload(w, storage="f32")
    b = lbpf.sim_from_workload(w, storage="f32")
    b.set_schedule("one_launch")
    b.set_tiling(*tiling)
    a.step(14)
    b.step(14)
    _same(a, b)


def test_schedule_switches_mid_run():
    w = workloads.large_kh(n=64)
    a = lbpf.sim_from_workload(w, storage="f32")
    b = lbpf.sim_from_workload(w, storage="f32")
    a.step(20)
    b.step(7)
    b.set_schedule("one_launch")
    b.step(8)
    b.set_schedule("two_kernels")
    b.step(5)
    _same(a, b)


def test_batch_one_launch_matches_single_bitwise():
    ws = workloads.batch_sweep(count=5, storage="f16")
    singles = [lbpf.sim_from_workload(w) for w in ws]
    batch = lbpf.batch_from_workloads(ws)
    batch.set_schedule("one_launch")
    assert batch.schedule == "one_launch"
    batch.step(3)
    batch.step(12)
    for s in singles:
        s.step(15)
    for s, m in zip(singles, batch.sims):
        _same(s, m)
    batch.close()


def test_one_launch_autotune_keeps_state():
    w = workloads.coupled_dendrite(n=40)
    a = lbpf.sim_from_workload(w, storage="f32")
    b = lbpf.sim_from_workload(w, storage="f32")
    b.set_schedule("one_launch")
    a.step(5)
    b.step(5)
    assert b.autotune(steps=2) > 0
    assert b.schedule == "one_launch"
    a.step(7)
    b.step(7)
    _same(a, b)


def test_one_launch_refused_where_not_instantiated():
    s64 = lbpf.Sim((24, 20, 16), (19, 19, 0), storage="f64")
    with pytest.raises(lbpf.LbpfError) as e:
        s64.set_schedule("one_launch")
    assert e.value.code == lbpf.LBPF_EINVAL
    s15 = lbpf.Sim((24, 20, 16), (15, 19, 0), storage="f32")
    with pytest.raises(lbpf.LbpfError):
        s15.set_schedule("one_launch")
    assert s15.schedule == "two_kernels"


def test_bounded_wait_gives_up_and_device_stays_usable():
    assert lbpf.wait_probe(1, 1000) is True
    t0 = time.perf_counter()
    assert lbpf.wait_probe(0, 4000) is False  # a flag that nothing sets: the wait gives up
    assert time.perf_counter() - t0 < 5.0
    w = workloads.coupled_dendrite(n=32)
    s = lbpf.sim_from_workload(w, storage="f32")
    s.set_schedule("one_launch")
    s.step(6)
    assert np.all(np.isfinite(s.sums()))


def test_wait_that_gives_up_is_reported():
    """The failure path of the one-launch step without a hang: with each wait bounded to zero
    polls every U/theta tile gives up at once (nothing spins), sets the handle's flag and
    goes ahead; the next call that returns data reports LBPF_ETIMEOUT, the handle stays
    failed, and the device stays usable for another handle."""
    w = workloads.coupled_dendrite(n=32)
    s = lbpf.sim_from_workload(w, storage="f32")
    s.set_schedule("one_launch")
    s.set_wait_polls(0)
    s.step(6)
    with pytest.raises(lbpf.LbpfError) as e:
        s.sums()
    assert e.value.code == lbpf.LBPF_ETIMEOUT
    with pytest.raises(lbpf.LbpfError) as e:
        s.step(1)
    assert e.value.code == lbpf.LBPF_ETIMEOUT
    t = lbpf.sim_from_workload(w, storage="f32")
    t.set_schedule("one_launch")
    t.step(6)
    assert np.all(np.isfinite(t.sums()))


"""Temporal blocking: two BBK steps per launch (the band kernel) give the same
bits as one step per launch, through graph chunks and direct launches,
around recording steps, and for shapes it does not take (which keep one step
per launch).  The per-site arithmetic is shared, so the comparison is exact;
the one-step kernels are checked against the oracle elsewhere."""
import numpy as np
import pytest
import torch

from paper_2409_06412_gb300 import XY_PATH_BATCHED, XY_PATH_PLAIN, build
from tests import inputs
from tests.gpu_helpers import make_pair

pytestmark = pytest.mark.gpu
TC = inputs.T_C

# (Lx, Ly, replicas): two-step shapes (2, 4, 8 and 3 warps wide; one band of
# 8 rows whose halos are its own rows), beside shapes it does not take
SHAPES = [(256, 64, 3), (512, 32, 2), (1024, 16, 1), (384, 24, 1), (256, 8, 2), (64, 64, 1), (12, 10, 1),
          (128, 32, 2)]
STRIP2 = 6  # timing class of the two-step launches


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()


def _specs(totals=None, T=TC):
    return [inputs.config(Lx, Ly, n, seed=11 + i, knots=([0], [T]),
                          n_total=(totals[i] if totals else 10 ** 9))
            for i, (Lx, Ly, n) in enumerate(SHAPES)]


def _pair(specs, seed=3):
    thetas = [inputs.angles(s["n_rep"], s["Lx"], s["Ly"], seed + i) for i, s in enumerate(specs)]
    two, _, _ = make_pair(specs, thetas, path=XY_PATH_BATCHED)
    two.set_temporal_blocking(2)
    ref, _, _ = make_pair(specs, thetas, path=XY_PATH_PLAIN)
    return two, ref


def _same(a, b):
    torch.cuda.synchronize()
    return torch.equal(a.theta, b.theta) and torch.equal(a.omega, b.omega)


def test_two_steps_per_launch_are_bit_identical():
    two, ref = _pair(_specs())
    for n in (37, 40, 96, 4, 3):  # odd and even calls, whole 32-step graph chunks, a lone pair batch
        two.step(n)
        ref.step(n)
        assert _same(two, ref), n
    # the same through direct launches, with the launches counted
    two.set_kernel_timing(True)
    two.step(64)
    ms, launches = two.kernel_timing()
    two.set_kernel_timing(False)
    ref.step(64)
    assert _same(two, ref)
    assert launches[STRIP2] > 0 and ms[STRIP2] > 0, launches
    # back to one step per launch mid-run: the state is where single steps leave it
    two.set_temporal_blocking(1)
    two.step(33)
    ref.step(33)
    assert _same(two, ref)


@pytest.mark.parametrize("every", [50, 8])
def test_two_steps_around_recording_steps(every):
    """Records every 50 steps (the stretches between them run two steps per
    launch) and every 8 (chunks that record run one step per launch): the
    same states and the same records as one step per launch."""
    specs = _specs(T=1.2)
    two, ref = _pair(specs, seed=5)
    one, _ = _pair(specs, seed=5)
    one.set_temporal_blocking(1)
    for lat in (two, one, ref):
        lat.step(7)
    r2 = two.step(130, record_every=every)
    r1 = one.step(130, record_every=every)
    ref.step(130, record_every=every)
    assert _same(two, ref) and _same(one, ref)
    torch.cuda.synchronize()
    assert torch.equal(torch.nan_to_num(r2, nan=7.0), torch.nan_to_num(r1, nan=7.0))


def test_uneven_lengths_keep_one_step_per_launch():
    """Configurations of one shape that end at different steps: no pair may
    straddle a last step, so that shape runs one step per launch for the call,
    and the result is the same as the plain path's."""
    totals = [90, 41, 200, 10 ** 9, 60, 77, 5, 100]
    two, ref = _pair(_specs(totals), seed=7)
    two.set_kernel_timing(True)
    two.step(150)
    ms, launches = two.kernel_timing()
    ref.step(150)
    assert _same(two, ref)
    _, steps = two.observe()
    assert list(steps) == [min(t, 150) for t in totals]
    # every two-step shape here has configurations of unequal length except
    # (1024, 16) and (384, 24), which still pair up
    assert launches[STRIP2] > 0


def test_two_steps_with_a_field_schedule():
    """The two-step kernel takes each step's own field (h_k and h_{k+1} of a
    ramp): the same bits as one step per launch."""
    specs = [dict(s, field=([0, 60], [0.4, 2.2])) for s in _specs()]
    two, ref = _pair(specs, seed=9)
    for n in (64, 36):
        two.step(n)
        ref.step(n)
    assert _same(two, ref)


def test_two_steps_with_coupling_profiles():
    """The two-step kernel takes each step's own couplings (J_par a(k),
    J_perp b(k) of an anisotropic ramp): the same bits as one step per launch."""
    specs = [dict(s, couplings=([0, 60], [1.0, 0.4], [0.5, 2.5])) for s in _specs()]
    two, ref = _pair(specs, seed=10)
    for n in (64, 36):
        two.step(n)
        ref.step(n)
    assert _same(two, ref)


def test_temporal_blocking_rejects_bad_modes():
    from paper_2409_06412_gb300 import XYError
    two, _ = _pair(_specs())
    with pytest.raises(XYError):
        two.set_temporal_blocking(3)
    with pytest.raises(XYError):
        two.set_temporal_blocking(-1)

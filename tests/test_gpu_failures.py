"""Failure detection without a GPU fault: every device-side wait in libmach
is bounded, gives up after its poll limit, records a status bit and returns,
and the call reports MACH_ETIMEOUT with the context still usable
(mach_check_bounded_wait runs that wait with a short limit on a barrier that
nothing completes)."""
import numpy as np
import pytest

from tests._gpu import mach_module, torch

pytestmark = pytest.mark.gpu


def test_bounded_wait_completes_when_the_barrier_does():
    mach = mach_module()
    assert mach.check_bounded_wait(1 << 16, True) == 0


def test_bounded_wait_times_out_and_the_context_survives():
    mach = mach_module()
    assert mach.check_bounded_wait(2000, False) == 5          # MACH_ETIMEOUT
    assert mach.check_bounded_wait(1, False) == 5
    # the device context is intact: a sampler call afterwards succeeds
    x = torch.randn(20, 30, 40, device="cuda")
    s = mach.sample(x, 0.5, 3)
    assert 0 < s.count() < x.numel()
    s.free()
    torch.cuda.synchronize()


def test_bounded_wait_rejects_bad_limits():
    mach = mach_module()
    assert mach.check_bounded_wait(0, False) == 1             # MACH_EINVAL
    assert mach.check_bounded_wait((1 << 23) + 1, False) == 1

"""GPU parity of Tucker2 (mach_hooi_tucker2: one mode kept whole, Section 2.1
Tucker-n and the Tucker2 of Section 4) against the FP64 oracle: subspaces,
sign-fixed core and reconstruction error within 1e-10 (FP64) and 1e-5
(FP32), for each choice of the kept mode, with the small-Gram routes on both
sides (r_other * I_keep above and below I_n)."""
import numpy as np
import pytest

from oracle import mach_oracle as O
from paper_0909_4969_gb300 import synth
from tests._gpu import compare_decomposition, mach_module, torch

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}
# FP32: the sign-fixed core is compared where the core singular-value gaps
# g satisfy 2^-22 / g <= 1e-5 (below that FP32 does not fix the individual
# singular vectors to 1e-5; subspaces and reconstruction error are compared
# in every case)
ROUNDING = {"fp64": None, "fp32": 2.0 ** -22}


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("dims,ranks,keep,p", [
    ((30, 6, 400), (4, 3, 0), 2, 0.3),      # long kept mode (time-like): both Grams I_n x I_n
    ((5, 40, 60), (0, 4, 5), 0, 0.4),       # short kept mode: both Grams r_other I_keep square
    ((50, 7, 45), (4, 0, 3), 1, 0.3),       # kept middle mode
])
def test_tucker2_matches_oracle(dims, ranks, keep, p, prec):
    mach = mach_module()
    true_ranks = tuple(min(dims[k], 4) if k == keep else r for k, r in enumerate(ranks))
    X, _, _ = synth.tucker_numpy(synth.TuckerSpec(dims, true_ranks, "gaussian", 0.05, 9, "float64"))
    S, G_o, A_o = O.mach_tucker2(X, ranks, keep, p, 17, 8)
    s = mach.sample(torch.from_numpy(X).cuda(), p, 17)
    G_g, A_g = s.tucker2(ranks, keep, 8, prec)
    torch.cuda.synchronize()
    assert s.stats()["flags"] == 0
    assert A_g[keep] is None                      # the kept mode's factor is the identity
    A_g = [np.eye(dims[k]) if a is None else a.cpu().numpy() for k, a in enumerate(A_g)]
    assert G_g.shape == G_o.shape
    r = compare_decomposition(O, X, G_o, A_o, G_g.cpu().numpy(), A_g, TOL[prec], "tucker2 %s keep %d" % (prec, keep),
                              rounding=ROUNDING[prec])
    s.free()
    _CORE_COUNT[prec] = _CORE_COUNT.get(prec, 0) + int(r["core_compared"])
    _CORE_COUNT[prec + "_n"] = _CORE_COUNT.get(prec + "_n", 0) + 1


_CORE_COUNT = {}


def test_tucker2_core_was_compared():
    """The FP32 cases above compare the sign-fixed core only where the core's
    singular-value gaps allow it: at least one of them must have done so
    (the FP64 cases always do)."""
    if not _CORE_COUNT:
        pytest.skip("the Tucker2 parity cases did not run")
    print("tucker2 core compared:", _CORE_COUNT)
    assert _CORE_COUNT.get("fp64", 0) == _CORE_COUNT.get("fp64_n", 0)
    assert _CORE_COUNT.get("fp32", 0) >= 1, _CORE_COUNT


def test_tucker2_rejects_bad_arguments():
    mach = mach_module()
    s = mach.sample(torch.randn(20, 10, 30, device="cuda", dtype=torch.float64), 0.5, 3)
    with pytest.raises(mach.MachError):
        s.tucker2((4, 3, 0), 3, 2, "fp64")          # no mode 3
    with pytest.raises(mach.MachError):
        s.tucker2((25, 3, 0), 2, 2, "fp64")         # r_0 > I_0
    x4 = mach.sample(torch.randn(5, 6, 7, 8, device="cuda"), 0.5, 3)
    with pytest.raises(mach.MachError):
        x4.tucker2((2, 2, 2, 0), 3, 2, "fp32")      # not 3-way
    s.free()
    x4.free()

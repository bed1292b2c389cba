"""The HOSVD Gram X^_(n) X^_(n)^T of the sampled tensor (mach_sample_gram)
against the oracle's sparse Gram of the same kept entries: the exact FP64
route within rounding, and the tensor-core routes (BF16 values, FP32
accumulation) within their stated precision, on shapes that cover one and
several 256 x 256 blocks, ragged block edges, several chunk ranges per
block and both value types."""
import numpy as np
import pytest

from oracle import mach_oracle as O
from paper_0909_4969_gb300 import synth
from tests._gpu import mach_module, torch

pytestmark = pytest.mark.gpu

# relative Frobenius error of the Gram: one BF16 rounding per value
# (2^-9 relative) for method 1; a BF16 pair (about 2^-17) for method 2
TOL = {0: 1e-12, 1: 8e-3, 2: 1e-4}


@pytest.mark.parametrize("dims,p,dtype", [
    ((200, 60, 70), 0.05, "float32"),       # I_0 = 200: one block
    ((300, 40, 50), 0.1, "float64"),        # I_0 = 300: 2 x 2 blocks, ragged
    ((1000, 24, 30), 0.2, "float32"),       # I_0 = 1000: 4 x 4 blocks
    ((7, 500, 90), 0.3, "float32"),         # tiny order, many fibres
])
def test_gram_methods_match_oracle(dims, p, dtype):
    mach = mach_module()
    X, _, _ = synth.tucker_numpy(synth.TuckerSpec(dims, (3, 3, 3), "gaussian", 0.1, 4, dtype))
    S = O.SampledTensor(X.shape, *O.sample(X, p, 77), p)
    s = mach.sample(torch.from_numpy(X).cuda(), p, 77)
    for mode in range(3):
        ref = S.gram(mode)
        nref = np.linalg.norm(ref)
        for method in (0, 1, 2):
            G = s.gram(mode, method).cpu().numpy()
            if method > 0:
                assert np.array_equal(G, G.T), (mode, method)     # symmetrised by construction
            else:
                assert np.max(np.abs(G - G.T)) <= 1e-14 * np.max(np.abs(G)), mode   # pair sums in any order
            rel = np.linalg.norm(G - ref) / nref
            assert rel <= TOL[method], "mode %d method %d: relative error %.3e" % (mode, method, rel)
    torch.cuda.synchronize()
    assert s.stats()["flags"] == 0
    s.free()


def test_gram_rejects_bad_arguments():
    mach = mach_module()
    s = mach.sample(torch.randn(20, 30, 40, device="cuda"), 0.5, 1)
    for mode, method in ((3, 0), (0, 3), (-1, 1)):
        with pytest.raises(mach.MachError):
            s.gram(mode, method)
    s.free()

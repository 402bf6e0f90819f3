"""Host-side pieces of the learned closure that need no GPU: the library's
order-transfer matrices (modal truncation in the orthogonal basis) against
the oracle's restriction (monomial Gram matrices, exact arithmetic), and
the sizes of the network's parameter vector and workspace."""
import numpy as np
import pytest

from oracle import closure
from paper_1409_0405_gb300 import fr


@pytest.mark.parametrize("etype", ["tet", "pri", "hex"])
@pytest.mark.parametrize("p_hi,p_lo", [(4, 2), (3, 1), (4, 3), (2, 1)])
def test_restriction_matches_oracle(etype, p_hi, p_lo):
    R = fr.transfer(etype, p_hi, p_lo)
    Ro = closure.restriction(etype, p_hi, p_lo)
    assert R.shape == Ro.shape
    np.testing.assert_allclose(R, Ro, rtol=0, atol=1e-13)


@pytest.mark.parametrize("etype", ["tet", "pri", "hex"])
def test_prolongation_then_restriction_is_identity(etype):
    up = fr.transfer(etype, 2, 4)
    down = fr.transfer(etype, 4, 2)
    np.testing.assert_allclose(down @ up, np.eye(down.shape[0]), atol=1e-13)
    # the prolongation is the interpolation of the p=2 polynomial: p=2
    # points of the p=4 space evaluate it back unchanged through M0-like
    # consistency, and a constant stays a constant
    np.testing.assert_allclose(up @ np.ones(up.shape[1]), np.ones(up.shape[0]), atol=1e-14)


def test_transfer_same_order_is_identity():
    for et in ("tet", "pri", "hex"):
        np.testing.assert_allclose(fr.transfer(et, 3, 3), np.eye(fr.transfer(et, 3, 3).shape[0]), atol=1e-14)


def test_transfer_rejects_bad_arguments():
    with pytest.raises(fr.FRError):
        fr.transfer("tet", 5, 2)
    with pytest.raises(fr.FRError):
        fr.transfer(3, 4, 2)


def test_mlp_sizes():
    nin, nh, nout = 360, 128, 90
    assert fr.mlp_nparams(nin, nh, nout) == nh * nin + nh + nh * nh + nh + nout * nh + nout
    ws = fr.mlp_workspace(nin, nh, nout, 1000)
    assert ws >= 1000 * (6 * nh + 2 * nout)
    assert fr.mlp_nparams(0, nh, nout) == 0

"""Host-side dense SIFT plan (no GPU needed): the descriptor count the
library derives for an image size and parameters equals the oracle's grid
over the same pyramid, and parameters outside their ranges are refused."""
import pytest

from oracle import dsift_oracle as O
from paper_1604_03498_gb300 import fv


@pytest.mark.parametrize("H,W,b,S,n,top", [(240, 320, 4, 4, 8, 1), (57, 83, 4, 4, 8, 1), (240, 320, 8, 4, 8, 1),
                                           (100, 130, 4, 2, 9, 2), (16, 16, 4, 4, 1, 0), (15, 400, 4, 4, 8, 1),
                                           (480, 640, 6, 3, 5, 1)])
def test_count_matches_oracle_grid(H, W, b, S, n, top):
    got = fv.fv_dsift_count(H, W, bin_size=b, stride=S, n_scales=n, top_scale=top)
    assert got == O.count(H, W, b, S, n, top)


@pytest.mark.parametrize("kw", [dict(bin_size=3), dict(bin_size=4, stride=3), dict(n_scales=0), dict(n_scales=10),
                                dict(bin_size=18)])
def test_bad_parameters_are_refused(kw):
    with pytest.raises(fv.FVError) as e:
        fv.fv_dsift_count(240, 320, **kw)
    assert e.value.status == fv.FV_ERR_INVALID

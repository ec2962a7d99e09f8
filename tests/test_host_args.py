"""Host-side argument handling of the Python binding (no GPU): the patch array that LBSim
hands to lb_create."""
import pytest

from paper_1704_03172_gb300 import lbac
from paper_1704_03172_gb300.sim import patch_array


def test_single_patch_defaults():
    a = patch_array((10, 12, 20, 22))
    assert len(a) == 1
    p = a[0]
    assert (p.x0, p.y0, p.nx_c, p.ny_c, p.ratio, p.coupling) == (10, 12, 20, 22, 2,
                                                                  lbac.LB_COUPLE_BOTH)


def test_nested_patches_with_one_coupling_each():
    a = patch_array([(10, 12, 20, 22), (4, 5, 8, 9, 2)], ["c2f", "f2c"])
    assert len(a) == 2
    assert [p.coupling for p in a] == [lbac.LB_COUPLE_C2F, lbac.LB_COUPLE_F2C]
    assert (a[1].x0, a[1].y0, a[1].nx_c, a[1].ny_c) == (4, 5, 8, 9)


def test_one_coupling_value_applies_to_every_patch():
    a = patch_array([(10, 12, 20, 22), (4, 5, 8, 9)], "f2c")
    assert [p.coupling for p in a] == [lbac.LB_COUPLE_F2C] * 2


@pytest.mark.parametrize("patch,coupling", [
    ((1, 1, 2, 2), "sideways"),
    ([(1, 1, 2, 2), (3, 3, 4, 4)], ["c2f"]),          # one value for two patches
    ([(1, 1, 2, 2)], ["c2f", "f2c"]),                  # two values for one patch
])
def test_bad_coupling_is_refused(patch, coupling):
    with pytest.raises(ValueError):
        patch_array(patch, coupling)

"""The slab plan of the host-buffer step (cdi_step_host for nz >= 16), host arithmetic only:
the slabs cover the planes, every slab holds the two halo planes, the copy-in pieces (after
the two seam planes) cover every plane, and by the time piece j has landed every plane that
slab j's step reads -- its planes and two more on either side, periodic in z -- has landed."""
import pytest

from paper_1803_01262_gb300 import build as B
from paper_1803_01262_gb300 import cdi


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    return cdi.lib()


@pytest.mark.parametrize("nz", list(range(16, 80)) + [127, 128, 255, 256, 257, 511, 512, 1000, 1024, 4097])
def test_plan_covers_and_lands_halos_first(nz):
    b, lo, hi = cdi.host_slab_plan(nz)
    assert b[0] == 0 and b[8] == nz
    assert all(b[j + 1] - b[j] >= 2 for j in range(8))
    landed = set(range(nz - 2, nz))          # the seam planes go first
    for j in range(8):
        assert 0 <= lo[j] and hi[j] <= nz
        landed |= set(range(lo[j], hi[j]))
        need = {z % nz for z in range(b[j] - 2, b[j + 1] + 2)}
        assert need <= landed, (j, sorted(need - landed))
    assert landed == set(range(nz))


def test_plan_refusals():
    with pytest.raises(cdi.CDIError) as e:
        cdi.host_slab_plan(15)
    assert e.value.code == cdi.CDI_ERR_DIM
    assert cdi.lib().cdi_host_slab_plan(64, None, None, None) == cdi.CDI_ERR_ARG

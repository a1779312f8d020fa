"""dm_legendre_analysis_noalloc: the Legendre analysis for callers that must
not allocate device memory when they call it (stream capture into a CUDA
graph, real-time loops where cudaMalloc could synchronise the device, hosts
that fix the library's memory budget).  It must give the same coefficients as
dm_legendre_analysis, call after call, with its scratch in the fixed
file-scope array.  This file is collected last so that a run stopping at the
first failure has already run every other test."""
import numpy as np
import pytest

from tests.gpu_helpers import alm_dev, rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1801_05358_gb300 import dmwf  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def test_noalloc_matches_analysis_on_two_calls():
    nside, lmax, B = 16, 40, 3
    rng = np.random.default_rng(7)
    shape = (B, 3, 4 * nside - 1, lmax + 1)
    p = dmwf.Plan(nside, lmax, B)
    outs = []
    for call in range(2):
        rc = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
        ref = torch.zeros((B, 3, (lmax + 1) * (lmax + 2) // 2, 2), dtype=torch.float64, device="cuda")
        got = torch.full_like(ref, float("nan"))
        p.legendre_analysis(alm_dev(rc), ref)
        p.legendre_analysis_noalloc(alm_dev(rc), got)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert rel(g, r) < 1e-12, call
        outs.append(g)
    assert rel(outs[0], outs[1]) > 1e-3  # the second call really recomputed


def test_noalloc_rejects_plans_beyond_its_scratch():
    p = dmwf.Plan(256, 512, 2)  # needs 2 x 8 x 3 x 131841 x 16 bytes > 64 MiB
    rc = torch.zeros((2, 3, 4 * 256 - 1, 513, 2), dtype=torch.float64, device="cuda")
    alm = torch.zeros((2, 3, 513 * 514 // 2, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(dmwf.DmError) as ei:
        p.legendre_analysis_noalloc(rc, alm)
    assert ei.value.status == dmwf.DM_EINVAL
    assert "scratch" in str(ei.value)

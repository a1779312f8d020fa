"""dm_legendre_analysis_noalloc: the Legendre analysis for callers that must
not allocate device memory when they call it (stream capture into a CUDA
graph, real-time loops where cudaMalloc could synchronise the device, hosts
that fix the library's memory budget).  It must give the same coefficients as
dm_legendre_analysis and as the oracle's analysis, call after call, with its
scratch in the fixed file-scope array:
- at sizes with one and with several chunks of 64 ring pairs (the per-chunk
  partial sums and their reduction), and with polar seeds below 2^-600 (the
  rescaled region of the recurrence: nside 64 / lmax 128 and nside 256 /
  lmax 512 both reach it);
- inside a captured CUDA graph, replayed on new inputs, and without any
  change of the device's free memory across a call.
This file is collected last so that a run stopping at the first failure has
already run every other test."""
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


def _rc(rng, B, nside, lmax):
    shape = (B, 3, 4 * nside - 1, lmax + 1)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def _alm_buf(B, lmax, fill=0.0):
    return torch.full((B, 3, (lmax + 1) * (lmax + 2) // 2, 2), fill, dtype=torch.float64, device="cuda")


def test_noalloc_matches_analysis_on_two_calls():
    nside, lmax, B = 16, 40, 3
    rng = np.random.default_rng(7)
    p = dmwf.Plan(nside, lmax, B)
    outs = []
    for call in range(2):
        rc = _rc(rng, B, nside, lmax)
        ref = _alm_buf(B, lmax)
        got = _alm_buf(B, lmax, float("nan"))
        p.legendre_analysis(alm_dev(rc), ref)
        p.legendre_analysis_noalloc(alm_dev(rc), got)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g))
        assert rel(g, r) < 1e-12, call
        outs.append(g)
    assert rel(outs[0], outs[1]) > 1e-3  # the second call really recomputed
    p.close()


@pytest.mark.parametrize("nside,lmax,B", [(64, 128, 2), (256, 512, 1)])
def test_noalloc_several_chunks_and_rescaled_seeds(orc, nside, lmax, B):
    """2 and 8 chunks of ring pairs; polar seeds carried as v 2^-S (S > 0).
    Two calls in a row, each against dm_legendre_analysis and the oracle."""
    rng = np.random.default_rng(11 + nside)
    p = dmwf.Plan(nside, lmax, B)
    for call in range(2):
        rc = _rc(rng, B, nside, lmax)
        ref = _alm_buf(B, lmax)
        got = _alm_buf(B, lmax, float("nan"))
        p.legendre_analysis(alm_dev(rc), ref)
        p.legendre_analysis_noalloc(alm_dev(rc), got)
        torch.cuda.synchronize()
        g = got.cpu().numpy().view(np.complex128)[..., 0]
        r = ref.cpu().numpy().view(np.complex128)[..., 0]
        assert np.all(np.isfinite(g))
        assert rel(g, r) < 1e-12, call
        assert rel(g[0], orc.legendre_analysis(nside, lmax, rc[0])) < 1e-12, call
    p.close()


def test_noalloc_in_a_captured_graph_allocates_nothing():
    """After one call outside capture (which looks up the scratch address),
    the call is recorded into a CUDA graph; replays on new inputs match
    dm_legendre_analysis, and a plain call leaves the device's free memory
    unchanged."""
    nside, lmax, B = 32, 64, 2
    rng = np.random.default_rng(23)
    p = dmwf.Plan(nside, lmax, B)
    rc_static = alm_dev(_rc(rng, B, nside, lmax))
    out_static = _alm_buf(B, lmax)
    p.legendre_analysis_noalloc(rc_static, out_static)  # first call on this device: before capture
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    p.legendre_analysis_noalloc(rc_static, out_static)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        p.legendre_analysis_noalloc(rc_static, out_static)
    for _ in range(2):
        rc = _rc(rng, B, nside, lmax)
        rc_static.copy_(alm_dev(rc))
        out_static.fill_(float("nan"))
        g.replay()
        ref = _alm_buf(B, lmax)
        p.legendre_analysis(rc_static, ref)
        torch.cuda.synchronize()
        assert np.all(np.isfinite(out_static.cpu().numpy()))
        assert rel(out_static.cpu().numpy(), ref.cpu().numpy()) < 1e-12
    del g
    p.close()


def test_noalloc_rejects_plans_beyond_its_scratch():
    p = dmwf.Plan(256, 512, 2)  # needs 2 x 8 x 3 x 131841 x 16 bytes > 64 MiB
    rc = torch.zeros((2, 3, 4 * 256 - 1, 513, 2), dtype=torch.float64, device="cuda")
    alm = torch.zeros((2, 3, 513 * 514 // 2, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(dmwf.DmError) as ei:
        p.legendre_analysis_noalloc(rc, alm)
    assert ei.value.status == dmwf.DM_EINVAL
    assert "scratch" in str(ei.value)
    p.close()

"""GPU parity of the L-BFGS step (nst_lbfgs_step) and of the bicubic initialisation
(nst_upsample_init) against the FP64 oracles."""
import numpy as np
import pytest
import torch

from oracle import bicubic, lbfgs
from paper_2212_13459_gb300 import native

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,m,steps", [(1000, 5, 25), (4099, 10, 12), (257, 3, 40)])
def test_lbfgs_iterates_match_oracle(n, m, steps):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((64, n)) / np.sqrt(n)
    d = rng.uniform(0.5, 2.0, size=n)
    b = rng.standard_normal(n)
    grad = lambda z: d * z + A.T @ (A @ z) - b        # strictly convex quadratic
    x_ref = np.zeros(n)
    opt = lbfgs.LBFGS(n, m)
    x_gpu = torch.zeros(n, dtype=torch.float32, device="cuda")
    st = native.LBFGS(n, m)
    for k in range(steps):
        # both sides get the gradient at their own iterate (FP32 on the device)
        g_ref = grad(x_ref)
        opt.step(x_ref, g_ref)
        g_dev = torch.from_numpy(grad(x_gpu.cpu().numpy().astype(np.float64)).astype(np.float32))
        st.step(x_gpu, g_dev.cuda())
    xg = x_gpu.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(xg - x_ref) <= 1e-4 * np.linalg.norm(x_ref)
    pairs, iters = st.info()
    assert iters == steps and pairs == min(m, len(opt.S))


def test_lbfgs_long_history_follows_oracle():
    """History 100 (the paper's first scale) filled and rolling: both sides receive the same
    gradient sequence (the oracle's trajectory on an ill-conditioned quadratic), which keeps
    FP32 storage from compounding through x -> g (simulated: 8e-5 after 110 steps)."""
    n, m, steps = 3001, 100, 110
    rng = np.random.default_rng(n)
    d = np.logspace(-3, 1, n)
    rng.shuffle(d)
    b = rng.standard_normal(n)
    x_ref = np.zeros(n)
    opt = lbfgs.LBFGS(n, m)
    x_gpu = torch.zeros(n, dtype=torch.float32, device="cuda")
    st = native.LBFGS(n, m)
    for _ in range(steps):
        g = d * x_ref - b
        opt.step(x_ref, g)
        st.step(x_gpu, torch.from_numpy(g.astype(np.float32)).cuda())
    assert len(opt.S) == m
    pairs, _ = st.info()
    assert pairs == m
    xg = x_gpu.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(xg - x_ref) <= 1e-3 * np.linalg.norm(x_ref)


def test_lbfgs_skips_pairs_without_curvature():
    """An indefinite quadratic: from the third pair on y^T s < 0 (well away from 0 relative to
    |s| |y|), so the pairs are skipped and the history stays at two pairs on both sides."""
    n, m, steps = 2000, 5, 8
    rng = np.random.default_rng(11)
    d = rng.uniform(-0.6, 2.0, size=n)
    b = rng.standard_normal(n)
    x_ref = np.zeros(n)
    opt = lbfgs.LBFGS(n, m)
    x_gpu = torch.zeros(n, dtype=torch.float32, device="cuda")
    st = native.LBFGS(n, m)
    for _ in range(steps):
        opt.step(x_ref, d * x_ref - b)
        xg = x_gpu.cpu().numpy().astype(np.float64)
        st.step(x_gpu, torch.from_numpy((d * xg - b).astype(np.float32)).cuda())
    assert len(opt.S) == 2
    pairs, _ = st.info()
    assert pairs == 2
    xg = x_gpu.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(xg - x_ref) <= 1e-4 * np.linalg.norm(x_ref)


def test_lbfgs_first_step():
    g = torch.tensor([3.0, -1.0, 0.5, 0.0], device="cuda")
    x = torch.zeros(4, device="cuda")
    st = native.LBFGS(4, 10)
    st.step(x, g)
    assert np.allclose(x.cpu().numpy(), -g.cpu().numpy() / 4.5, rtol=1e-6)


@pytest.mark.parametrize("h,w,H,W", [(13, 17, 26, 34), (1512, 2016, 3024, 4032), (7, 9, 15, 20)])
def test_upsample_matches_oracle(h, w, H, W):
    rng = np.random.default_rng(h * w)
    xs = rng.uniform(0, 1, size=(3, h, w)).astype(np.float32)
    out = torch.empty((3, H, W), device="cuda")
    native.upsample_init(torch.from_numpy(xs).cuda(), out)
    ref = bicubic.upsample(xs.astype(np.float64), H, W)
    got = out.cpu().numpy()
    if H * W > 10 ** 6:   # full size: sampled rows
        rows = rng.integers(0, H, size=64)
        assert np.abs(got[:, rows] - ref[:, rows]).max() <= 1e-5
    else:
        assert np.abs(got - ref).max() <= 1e-5


@pytest.mark.parametrize("npix,C,dtype", [(1000, 64, torch.float32), (70001, 512, torch.bfloat16),
                                          (300, 128, torch.bfloat16), (5000, 256, torch.float32)])
def test_gram_entry_matches_float64(npix, C, dtype):
    """nst_gram (the Gram engine of Eq. 4 on one flat feature matrix) against a float64 product."""
    g = torch.Generator(device="cuda").manual_seed(npix + C)
    V = torch.rand(npix, C, device="cuda", generator=g).to(dtype)
    G = torch.full((C, C), 3.0, dtype=torch.float64, device="cuda")
    native.gram(V, G)
    ref = V.double().T @ V.double()
    assert ((G - ref).norm() / ref.norm()).item() <= 1e-6
    assert torch.equal(G, G.T)


@pytest.mark.parametrize("h,w,H,W", [(37, 53, 18, 26), (4226, 5319, 1057, 1330), (16, 24, 4, 6)])
def test_downscale_matches_oracle(h, w, H, W):
    from oracle import area
    rng = np.random.default_rng(h + w)
    x = rng.uniform(0, 1, size=(3, h, w)).astype(np.float32)
    out = torch.empty((3, H, W), device="cuda")
    native.downscale(torch.from_numpy(x).cuda(), out)
    got = out.cpu().numpy()
    if h * w > 10 ** 6:   # full size: sampled rows, the oracle on those rows' footprints
        rows = rng.integers(0, H, size=16)
        full = area.downscale(x.astype(np.float64), H, W)
        assert np.abs(got[:, rows] - full[:, rows]).max() <= 2e-6
    else:
        assert np.abs(got - area.downscale(x.astype(np.float64), H, W)).max() <= 2e-6


def test_lbfgs_host_history_gives_identical_iterates():
    """History in mapped host memory (the paper's CPU-side history of the last scale, Section
    5.1): the same kernels on the same values, so the iterates are bit-identical."""
    n, m = 20001, 7
    rng = np.random.default_rng(5)
    d = torch.tensor(rng.uniform(0.5, 2.0, size=n), dtype=torch.float32, device="cuda")
    b = torch.tensor(rng.standard_normal(n), dtype=torch.float32, device="cuda")
    xs = []
    for host in (False, True):
        x = torch.zeros(n, device="cuda")
        st = native.LBFGS(n, m, host_history=host)
        for _ in range(15):
            st.step(x, d * x - b)
        xs.append(x.clone())
        st.close()
    assert torch.equal(xs[0], xs[1])

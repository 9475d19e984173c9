"""Per-voxel conductivity mode, the gradient of sigma_* and the torch.autograd
layer, against the FP64 oracle and central finite differences."""
import numpy as np
import pytest

from oracle import exact as X
from oracle import schemes as S
from synth import bernoulli_majority_mask, random_mask, square_array_mask

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_08289_gb300 as lib
    from paper_2001_08289_gb300 import build

    build.build()
    lib.load_library()
    return lib


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("scheme", ["ms", "em"])
@pytest.mark.parametrize("cplx", [False, True])
def test_per_voxel_sigma_iterates_match_oracle(L, prec, tol, scheme, cplx):
    rng = np.random.default_rng(3)
    shape = (32, 64)
    sig = 1.0 + 9.0 * rng.random(shape)
    if cplx:
        sig = sig + 2.0j * rng.random(shape)
    e = np.array([0.8, 0.6])
    s0 = (sig.real.min() + sig.real.max()) / 2 if scheme == "ms" else np.sqrt(sig.real.min() * sig.real.max())
    with L.Grid(np.zeros(shape, np.uint8)) as g:
        g.set_sigma_field(sig)
        r = g.solve(1.0, e, scheme=scheme, precision=prec, green="fd", tol=0.0, max_iter=10)
        E = r.field_numpy()
        assert r.packed == (not cplx)
    pb = S.Problem(np.zeros(shape, np.uint8), 1.0, e, "fd", sigma_field=sig, sigma0=s0)
    ref = S.solve(pb, scheme, tol=0.0, max_iter=10)
    rel = np.abs(r.hist_sigma - ref.hist_sigma) / np.abs(ref.hist_sigma)
    assert rel.max() < tol
    assert np.linalg.norm(E - ref.E) / np.linalg.norm(ref.E) < 10 * tol


def test_per_voxel_sigma_3d_and_rejections(L):
    rng = np.random.default_rng(4)
    shape = (16, 16, 32)
    sig = 1.0 + 4.0 * rng.random(shape)
    e = np.array([0.0, 0.0, 1.0])
    with L.Grid(np.zeros(shape, np.uint8)) as g:
        g.set_sigma_field(sig)
        r = g.solve(1.0, e, scheme="em", precision="fp64", green="trig", tol=0.0, max_iter=8)
        with pytest.raises(L.LsfftError):
            g.solve(1.0, e, scheme="em_sub", alpha=0.1, beta=10.0)
    ref = S.solve(S.Problem(np.zeros(shape, np.uint8), 1.0, e, "trig", sigma_field=sig,
                            sigma0=np.sqrt(sig.min() * sig.max())), "em", tol=0.0, max_iter=8)
    assert np.max(np.abs(r.hist_sigma - ref.hist_sigma) / np.abs(ref.hist_sigma)) < 1e-10


@pytest.mark.parametrize("s1", [20.0, 2.0 + 1.0j])
def test_gradient_matches_oracle_and_finite_differences(L, s1):
    import torch

    mask = square_array_mask(32)
    e = [1.0, 0.0]
    sd, Ed = X.direct_solve(mask, s1, e, "fd")
    g_ref = X.gradient_sigma_field(Ed, e)
    with L.Grid(mask) as g:
        r = g.solve(s1, e, scheme="em_sub", precision="fp64", green="fd", tol=1e-14, max_iter=2000,
                    alpha=0.17, beta=6.0)
        grad = torch.empty((32, 32), dtype=torch.complex128, device="cuda")
        d1, energy = g.gradient(r, e, grad.data_ptr())
        gf = grad.cpu().numpy()
    assert np.abs(gf - g_ref).max() < 1e-10 * np.abs(g_ref).max()
    assert abs(energy - sd) < 1e-11 * abs(sd)
    h = 1e-4
    fd = (X.direct_solve(mask, s1 + h, e, "fd")[0] - X.direct_solve(mask, s1 - h, e, "fd")[0]) / (2 * h)
    assert abs(d1 - fd) < 1e-7 * abs(fd)


def test_gradient_per_voxel_central_differences_3d(L):
    """The adjoint configuration in small: majority-filtered Bernoulli voxels,
    sigma = 1 + 19 chi, gradient at random voxels against central differences of
    the variational energy estimate from FP64 solves."""
    import torch

    n = 16
    mask = bernoulli_majority_mask(n, p=0.2, seed=5, threshold=10)
    sig = 1.0 + 19.0 * mask.astype(float)
    e = [1.0, 0.0, 0.0]
    opts = dict(scheme="em", precision="fp64", green="fd", tol=1e-15, max_iter=3000)
    rng = np.random.default_rng(6)
    voxels = [tuple(rng.integers(0, n, 3)) for _ in range(6)]
    with L.Grid(mask) as g:
        g.set_sigma_field(sig, sigma0=np.sqrt(20.0))
        r = g.solve(1.0, e, **opts)
        grad = torch.empty(mask.shape, dtype=torch.complex128, device="cuda")
        g.gradient(r, e, grad.data_ptr())
        gf = grad.cpu().numpy().real
        h = 1e-3
        for v in voxels:
            vals = []
            for sgn in (1, -1):
                sp = sig.copy()
                sp[v] += sgn * h
                g.set_sigma_field(sp, sigma0=np.sqrt(20.0))
                rr = g.solve(1.0, e, **opts)
                vals.append(g.gradient(rr, e)[1].real)
            fd = (vals[0] - vals[1]) / (2 * h)
            assert abs(fd - gf[v]) < 1e-4 * abs(gf[v]) + 1e-13, (v, fd, gf[v])


def test_autograd_functions(L):
    import torch

    from paper_2001_08289_gb300 import autograd as AG

    mask = square_array_mask(32)
    e = [1.0, 0.0]
    with L.Grid(mask) as g:
        opts = dict(scheme="em_sub", precision="fp64", green="fd", tol=1e-14, max_iter=2000, alpha=0.17, beta=6.0)
        s1 = torch.tensor(20.0, dtype=torch.float64, requires_grad=True)
        out = AG.sigma_star(s1, g, e, **opts)
        out.backward()
        sd = X.direct_solve(mask, 20.0, e, "fd")[0].real
        assert abs(out.item() - sd) < 1e-11
        h = 1e-4
        fd = (X.direct_solve(mask, 20.0 + h, e, "fd")[0] - X.direct_solve(mask, 20.0 - h, e, "fd")[0]).real / (2 * h)
        assert abs(s1.grad.item() - fd) < 1e-7 * abs(fd)

        sig = torch.tensor(1.0 + 19.0 * mask, dtype=torch.float64, device="cuda", requires_grad=True)
        out = AG.sigma_star_field(sig, g, e, scheme="em", precision="fp64", green="fd", tol=1e-14, max_iter=3000)
        out.backward()
        _, Ed = X.direct_solve(mask, 20.0, e, "fd")
        ref = X.gradient_sigma_field(Ed, e).real
        assert np.abs(sig.grad.cpu().numpy() - ref).max() < 1e-9 * np.abs(ref).max()

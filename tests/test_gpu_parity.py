"""GPU parity: the CUDA path through the C ABI against the FP64 oracle.

Tolerances (stated for the task's targets): FP64 mode, sigma_k relative error
<= 1e-10 at every iterate and E relative L2 <= 1e-10; FP32 mode (complex FP32
fields, FP64 reductions), sigma_k relative error <= 1e-5 at every iterate and
E relative L2 <= 1e-4.  Runs use tol = 0 and a fixed number of updates so that
the histories align element by element; separate tests check the stop rule.
"""
import numpy as np
import pytest

from oracle import exact as X
from oracle import schemes as S
from synth import laminate_mask, random_mask, square_array_mask

pytestmark = pytest.mark.gpu

TOL = {"fp64": (1e-10, 1e-10), "fp32": (1e-5, 1e-4)}
AB = (0.25, 4.0)


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


def _compare(L, mask, s1, e, scheme, green, prec, iters, ab=AB, stol=None, etol=None):
    st, et = TOL[prec]
    st = stol or st
    et = etol or et
    with L.Grid(mask) as g:
        r = g.solve(s1, e, scheme=scheme, precision=prec, green=green, tol=0.0, max_iter=iters,
                    alpha=ab[0], beta=ab[1], check_every=4)
        E = r.field_numpy()
    ref = S.solve(S.Problem(mask, s1, e, green), scheme, alpha=ab[0], beta=ab[1], tol=0.0, max_iter=iters)
    assert r.status == L.ENOTCONV and r.iterations == iters
    assert len(r.hist_sigma) == len(ref.hist_sigma) == iters + 1
    rel = np.abs(r.hist_sigma - ref.hist_sigma) / np.abs(ref.hist_sigma)
    assert rel.max() < st, (scheme, green, prec, rel.max())
    nrel = np.abs(r.hist_field_norm - ref.hist_field_norm) / np.abs(ref.hist_field_norm)
    assert nrel.max() < max(st, 1e-9) * 10, nrel.max()
    erel = np.linalg.norm(E - ref.E) / np.linalg.norm(ref.E)
    assert erel < et, (scheme, green, prec, erel)
    np.testing.assert_allclose(r.mean_E, ref.mean_E, atol=10 * st * np.abs(ref.mean_E).max())
    return r, ref


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("green", ["trig", "fd"])
@pytest.mark.parametrize("scheme", ["ms", "em", "ms_sub", "em_sub"])
def test_parity_2d_square_array(L, scheme, green, prec):
    _compare(L, square_array_mask(64), 10.0, np.array([1.0, 0.0]), scheme, green, prec, 20)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme", ["ms", "em", "ms_sub", "em_sub"])
def test_parity_2d_complex_sigma_random_mask_nonsquare(L, scheme, prec):
    """Non-square grid (x 128, y 32), random mask, complex sigma_1 and tilted e."""
    mask = random_mask((32, 128), 0.3, seed=21)
    _compare(L, mask, 3.0 + 4.0j, np.array([0.6, 0.8]), scheme, "fd", prec, 15, ab=(0.01, 100.0))


@pytest.mark.parametrize("n", [16, 32, 256])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_parity_2d_sizes(L, n, prec):
    for scheme in ("ms", "em_sub"):
        _compare(L, square_array_mask(n), 100.0, np.array([1.0, 0.0]), scheme, "trig", prec, 10)


@pytest.mark.parametrize("shape", [(16, 8192), (8192, 16), (32, 4096), (4096, 32), (64, 2048), (2048, 64),
                                   (1024, 1024)])
def test_parity_2d_long_lines(L, shape):
    """Thin grids put every line length up to 8192 on both the row and the strided
    pass (the kernels with the largest shared-memory and register footprints)."""
    mask = random_mask(shape, 0.25, seed=sum(shape))
    e = np.array([1.0, 0.0])
    precs = ["fp32"] + (["fp64"] if shape[1] <= 4096 else [])
    for prec in precs:
        for scheme in ("ms", "em_sub"):
            _compare(L, mask, 10.0, e, scheme, "fd", prec, 6, ab=(0.05, 20.0))


@pytest.mark.parametrize("shape", [(8192, 16), (4096, 32), (2048, 64)])
def test_parity_long_columns_complex_sigma(L, shape):
    """Long columns with complex sigma_1 (complex layout on the cluster strided pass)."""
    mask = random_mask(shape, 0.3, seed=shape[0])
    e = np.array([0.6, 0.8])
    precs = ["fp32", "fp64"]
    for prec in precs:
        for scheme in ("ms", "em_sub"):
            _compare(L, mask, 2.0 + 1.5j, e, scheme, "fd", prec, 6, ab=(0.05, 20.0))
            _compare(L, mask, 2.0 + 1.5j, e, scheme, "trig", prec, 4, ab=(0.05, 20.0))


def test_fp64_rejects_8192_point_rows(L):
    """FP64 supports rows (x lines) up to 4096 points (shared-memory bound of the
    row pass); 8192-point columns run on the cluster strided pass."""
    with L.Grid(np.zeros((16, 8192), np.uint8)) as g:
        with pytest.raises(L.LsfftError) as ei:
            g.solve(2.0, [1.0, 0.0], precision="fp64")
        assert ei.value.status == L.EINVAL


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme", ["ms", "em", "ms_sub", "em_sub"])
def test_parity_3d(L, scheme, prec):
    mask = square_array_mask(16, d=3)
    _compare(L, mask, 5.0, np.array([1.0, 0.0, 0.0]), scheme, "trig", prec, 10)


def test_parity_3d_512_lines(L):
    """Line length 512 on all three axes' kernels via thin 3-D grids."""
    for shape in ((16, 16, 512), (16, 512, 16), (512, 16, 16)):
        mask = random_mask(shape, 0.2, seed=7)
        for prec in ("fp32", "fp64"):
            _compare(L, mask, 5.0, np.array([1.0, 0.0, 0.0]), "ms", "trig", prec, 5)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_parity_3d_nonuniform_grid_fd(L, prec):
    mask = random_mask((16, 32, 64), 0.2, seed=5)   # n = (64, 32, 16)
    for scheme in ("ms", "em_sub"):
        _compare(L, mask, 20.0, np.array([0.0, 0.0, 1.0]), scheme, "fd", prec, 8, ab=(0.02, 50.0))


@pytest.mark.parametrize("s1", [0.01, 1.0e4])
def test_parity_extreme_contrast(L, s1):
    for scheme in ("ms", "em", "em_sub"):
        _compare(L, square_array_mask(32), s1, np.array([1.0, 0.0]), scheme, "fd", "fp64", 12)


def test_em_sub_at_sigma1_zero(L):
    """The paper's sigma_1 = 0 experiment: EM in H'' is defined there (Eq. J43)."""
    _compare(L, square_array_mask(64), 0.0, np.array([1.0, 0.0]), "em_sub", "trig", "fp64", 20)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_converged_solution_matches_direct_solve(L, prec):
    mask = square_array_mask(32)
    e = np.array([1.0, 0.0])
    sd, Ed = X.direct_solve(mask, 10.0, e, "fd")
    tol = 1e-13 if prec == "fp64" else 1e-7
    with L.Grid(mask) as g:
        for scheme in ("ms", "em", "ms_sub", "em_sub"):
            r = g.solve(10.0, e, scheme=scheme, precision=prec, green="fd", tol=tol, max_iter=2000,
                        alpha=0.17, beta=6.0)
            assert r.status == L.OK
            E = r.field_numpy()
            lim_s, lim_e = (1e-10, 1e-9) if prec == "fp64" else (1e-5, 1e-4)
            assert abs(r.sigma_star - sd) / abs(sd) < lim_s
            assert np.linalg.norm(E - Ed) / np.linalg.norm(Ed) < lim_e


def test_stop_rule_matches_oracle_fp64(L):
    mask = square_array_mask(64)
    e = np.array([1.0, 0.0])
    with L.Grid(mask) as g:
        for scheme in ("ms", "em", "em_sub"):
            r = g.solve(10.0, e, scheme=scheme, precision="fp64", green="trig", tol=1e-8, max_iter=500,
                        alpha=0.25, beta=4.0, check_every=3)
            ref = S.solve(S.Problem(mask, 10.0, e, "trig"), scheme, alpha=0.25, beta=4.0, tol=1e-8, max_iter=500)
            assert r.status == L.OK and ref.status == S.STATUS_OK
            assert r.iterations == ref.iterations
            assert abs(r.sigma_star - ref.sigma_star) < 1e-10 * abs(ref.sigma_star)


def test_laminate_exact_on_gpu(L):
    n, w, s1 = 64, 4, 7.0
    mask = laminate_mask((n, n), w, axis=0)
    f = mask.mean()
    with L.Grid(mask) as g:
        rx = g.solve(s1, [1.0, 0.0], scheme="em_sub", precision="fp64", green="trig", tol=1e-14, max_iter=500,
                     alpha=0.05, beta=20.0)
        ry = g.solve(s1, [0.0, 1.0], scheme="em_sub", precision="fp64", green="trig", tol=1e-14, max_iter=500,
                     alpha=0.05, beta=20.0)
    assert abs(rx.sigma_star - (f * s1 + 1 - f)) < 1e-11
    assert abs(ry.sigma_star - 1 / (f / s1 + 1 - f)) < 1e-11


def test_divergence_and_invalid_arguments(L):
    mask = square_array_mask(32)
    with L.Grid(mask) as g:
        r = g.solve(-2.0, [1.0, 0.0], scheme="ms", precision="fp64", tol=1e-8, max_iter=5000)
        assert r.status == L.EDIVERGED
        for kw in (dict(scheme="ms", s1=-1.0), dict(scheme="em", s1=0.0),
                   dict(scheme="em_sub", s1=1.0, alpha=0.0, beta=4.0),
                   dict(scheme="em_sub", s1=-0.25, alpha=0.25, beta=4.0),
                   dict(scheme="ms", s1=1.0, max_iter=0), dict(scheme="ms", s1=float("nan"))):
            s1 = kw.pop("s1")
            with pytest.raises(L.LsfftError) as ei:
                g.solve(s1, [1.0, 0.0], **kw)
            assert ei.value.status == L.EINVAL
        with pytest.raises(L.LsfftError):
            g.solve(1.0, [0.0, 0.0])


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_packed_real_layout_used_and_agrees_with_complex_layout(L, prec):
    """Real sigma_1 in 2-D runs the packed layout (E_x + i E_y in one plane); a
    negligible imaginary part forces the complex layout: the two must agree."""
    mask = random_mask((64, 128), 0.3, seed=3)
    e = [0.8, 0.6]
    with L.Grid(mask) as g:
        for scheme in ("ms", "em", "ms_sub", "em_sub"):
            kw = dict(scheme=scheme, precision=prec, green="fd", tol=0.0, max_iter=12, alpha=0.05, beta=20.0)
            rp = g.solve(10.0, e, **kw)
            rc = g.solve(complex(10.0, 1e-300), e, **kw)
            assert rp.packed and not rc.packed
            tol = 1e-12 if prec == "fp64" else 1e-6
            assert np.max(np.abs(rp.hist_sigma - rc.hist_sigma) / np.abs(rc.hist_sigma)) < tol
            Ep, Ec = rp.field_numpy(), rc.field_numpy()
            assert np.linalg.norm(Ep - Ec) / np.linalg.norm(Ec) < (1e-12 if prec == "fp64" else 1e-5)
    with L.Grid(square_array_mask(16, d=3)) as g:
        assert not g.solve(5.0, [1.0, 0.0, 0.0], max_iter=3, tol=0.0).packed


def test_field_tensor_is_a_zero_copy_view(L):
    """Result.field_tensor() wraps the result's device field without copying and
    keeps the result alive while the tensor is."""
    import gc

    import torch

    mask = square_array_mask(32)
    with L.Grid(mask) as g:
        r = g.solve(10.0, [1.0, 0.0], scheme="ms", precision="fp32", tol=0.0, max_iter=3)
        E = r.field_numpy()
        ptr = int(r._ptr.contents.E_device)
        t = r.field_tensor()
        assert t.is_cuda and t.dtype == torch.complex64 and tuple(t.shape) == E.shape
        assert t.data_ptr() == ptr
        del r
        gc.collect()
        np.testing.assert_array_equal(t.cpu().numpy(), E)
        del t
        gc.collect()


def test_async_field_copy_matches_the_synchronous_copy(L):
    """lsfft_copy_field_async delivers the same bytes as lsfft_copy_field, to
    pinned host memory and to device memory, while another solve runs on the
    grid's stream."""
    import torch

    mask = square_array_mask(64)
    with L.Grid(mask) as g:
        r1 = g.solve(10.0, [1.0, 0.0], scheme="ms", precision="fp32", tol=0.0, max_iter=5)
        E1 = r1.field_numpy()
        host = torch.empty(E1.shape, dtype=torch.complex64).pin_memory()
        dev = torch.empty(E1.shape, dtype=torch.complex64, device="cuda")
        cs = torch.cuda.Stream()
        r1.field_into_async(host.data_ptr(), False, cs.cuda_stream)
        r1.field_into_async(dev.data_ptr(), True, cs.cuda_stream)
        r2 = g.solve(0.1, [0.0, 1.0], scheme="em_sub", precision="fp32", tol=0.0, max_iter=5,
                     alpha=0.25, beta=4.0)
        cs.synchronize()
        np.testing.assert_array_equal(host.numpy(), E1)
        np.testing.assert_array_equal(dev.cpu().numpy(), E1)
        assert not np.array_equal(r2.field_numpy(), E1)
        r1.free()
        r2.free()
        with pytest.raises(ValueError):
            r1.field_into_async(host.data_ptr(), False, cs.cuda_stream)


def test_field_pool_reuses_and_returns_memory(L):
    """Workspaces and result fields come from a caching pool: repeated solves do
    not grow the device footprint, and once no grid or result is alive the
    pool hands its memory back to the driver."""
    import torch

    n = 4096
    field = 2 * n * n * 8                       # one complex FP32 [2][N] result field
    mask = square_array_mask(n)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    g = L.Grid(mask)
    try:
        for _ in range(2):
            g.solve(10.0, [1.0, 0.0], scheme="ms", precision="fp32", tol=0.0, max_iter=2).free()
        free1 = torch.cuda.mem_get_info()[0]
        for _ in range(6):
            g.solve(10.0, [1.0, 0.0], scheme="ms", precision="fp32", tol=0.0, max_iter=2).free()
        free2 = torch.cuda.mem_get_info()[0]
        assert abs(free2 - free1) < field // 4, (free1, free2)
        keep = [g.solve(10.0, [1.0, 0.0], scheme="ms", precision="fp32", tol=0.0, max_iter=2) for _ in range(3)]
        free3 = torch.cuda.mem_get_info()[0]
        assert free3 <= free2 - field, (free2, free3)   # two more live fields than before
        for r in keep:
            r.free()
    finally:
        g.close()
    torch.cuda.synchronize()
    free4 = torch.cuda.mem_get_info()[0]
    assert free4 >= free0 - 64 * 2**20, (free0, free4)

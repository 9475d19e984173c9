"""The split layout of long 2-D columns (n_x, n_y in {4096, 8192}, FP32 fields
with real coefficients): the row pass applies the first radix-2 step of every
y-DFT to row pairs (j, j + n_y/2) and the strided pass transforms independent
half-length columns.  Element by element against the FP64 oracle on 4096-point
grids (square and non-square, all four schemes, S and T of the substituted
schemes, a per-voxel conductivity), against the cluster layout at 8192^2, and
the layout switch."""
import numpy as np
import pytest

from oracle import schemes as S
from synth import random_mask, square_array_mask

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

ST, ET = 1e-5, 1e-4      # FP32 fields: sigma_k relative, E relative L2


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


def _compare(L, mask, s1, scheme, iters, e=(1.0, 0.0), green="trig", ab=(0.25, 4.0), sigma=None):
    e = np.array(e)
    with L.Grid(mask) as g:
        g.set_column_split(True)
        if sigma is not None:
            g.set_sigma_field(sigma)
        r = g.solve(s1, e, scheme=scheme, precision="fp32", green=green, tol=0.0, max_iter=iters,
                    alpha=ab[0], beta=ab[1])
        assert r.packed == 2, "the split layout did not run"
        E = r.field_numpy()
        hs = r.hist_sigma
        r.free()
    pb = S.Problem(mask, s1, e, green, sigma_field=sigma)
    ref = S.solve(pb, scheme, alpha=ab[0], beta=ab[1], tol=0.0, max_iter=iters)
    es = np.max(np.abs(hs - ref.hist_sigma) / np.abs(ref.hist_sigma))
    ee = np.linalg.norm(E - ref.E) / np.linalg.norm(ref.E)
    assert es < ST and ee < ET, (es, ee)


@pytest.mark.parametrize("scheme,s1,kind,green", [("ms", 10.0, "square", "trig"), ("em_sub", 10.0, "random", "trig"),
                                                  ("ms_sub", 0.1, "random", "fd"), ("em", 100.0, "square", "fd")])
def test_split_parity_4096(L, scheme, s1, kind, green):
    n = 4096
    mask = square_array_mask(n) if kind == "square" else random_mask((n, n), 0.3, seed=41)
    _compare(L, mask, s1, scheme, 3, e=(0.6, 0.8), green=green)


@pytest.mark.parametrize("shape", [(8192, 4096), (4096, 8192)])
def test_split_parity_non_square(L, shape):
    """n_y != n_x: the strided pass's half-length columns and the row pass's line
    length differ (8192 x 4096 runs 4096-point half-columns, 4096 x 8192 2048-point)."""
    mask = random_mask(shape, 0.25, seed=42)
    _compare(L, mask, 3.0, "em_sub", 2, e=(1.0, 0.0))


def test_split_per_voxel_conductivity(L):
    rng = np.random.default_rng(43)
    n = 4096
    sigma = 1.0 + 4.0 * rng.random((n, n))
    mask = np.zeros((n, n), np.uint8)
    _compare(L, mask, 1.0, "ms", 2, sigma=sigma)


def test_split_agrees_with_cluster_layout_8192(L):
    """Both strided-pass layouts of the 8192^2 square array give the same iterates
    up to FP32 rounding, and a converged sigma_* of EM in H''."""
    n = 8192
    mask = square_array_mask(n)
    out = {}
    with L.Grid(mask) as g:
        for split in (True, False):
            g.set_column_split(split)
            r = g.solve(10.0, [1.0, 0.0], scheme="em_sub", precision="fp32", tol=1e-6, max_iter=200,
                        alpha=0.25, beta=4.0)
            assert r.packed == (2 if split else 1) and r.status == L.OK
            out[split] = (r.hist_sigma.copy(), r.field_numpy(), r.iterations)
            r.free()
    (h1, E1, i1), (h0, E0, i0) = out[True], out[False]
    k = min(len(h1), len(h0))
    assert np.max(np.abs(h1[:k] - h0[:k]) / np.abs(h0[:k])) < 1e-6
    if i1 == i0:
        assert np.linalg.norm(E1 - E0) / np.linalg.norm(E0) < 1e-5

"""lsfft_autotune on the GPU: it times every candidate, returns a valid choice,
applies the layout to the grid, and solves with the tuned options agree with
untuned ones."""
import numpy as np
import pytest

from synth import square_array_mask

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


@pytest.mark.parametrize("n,candidates", [(256, 5), (4096, 10)])
def test_autotune_times_candidates_and_applies(L, n, candidates, tmp_path):
    from paper_2001_08289_gb300 import tune

    with L.Grid(square_array_mask(n)) as g:
        kw = dict(scheme="em_sub", precision="fp32", alpha=0.25, beta=4.0, tol=1e-6, max_iter=200)
        t = L.lsfft_autotune(g.handle, 10.0, [1.0, 0.0], L.make_opts(**kw), iters=16)
        assert t["candidates"] == candidates and t["check_every"] in (4, 8, 16, 32, 64)
        assert t["column_split"] in (0, 1) and t["ms_per_iter"] > 0
        if n < 4096:
            assert t["column_split"] == 0   # one layout exists: the default stays
        path = str(tmp_path / "tune.json")
        kw_t = tune.tuned(g, 10.0, [1.0, 0.0], path=path, **kw)
        r1 = g.solve(10.0, [1.0, 0.0], **kw_t)
        r0 = g.solve(10.0, [1.0, 0.0], **kw)
        assert r1.status == r0.status == L.OK
        assert abs(r1.sigma_star - r0.sigma_star) < 1e-6 * abs(r0.sigma_star)
        r1.free()
        r0.free()

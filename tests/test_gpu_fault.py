"""Bounded device waits: the TMA completion barriers of the strided passes give
up after a limit, the kernel records a fault and completes, and the solve
reports LSFFT_ECUDA; the GPU context stays usable.  The wait is made to run out
on purpose by the test hook lsfft_debug_inject (16 bytes announced to each
barrier that the copy never delivers), so no GPU fault is involved."""
import numpy as np
import pytest

from oracle import schemes as S
from synth import random_mask

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


# (4096, 16): 4096-point columns on the cluster pass; (64, 64): the plain strided pass
@pytest.mark.parametrize("shape", [(4096, 16), (64, 64)])
def test_bounded_tma_wait_reports_fault_and_recovers(L, shape):
    mask = random_mask(shape, 0.3, seed=3)
    e = [1.0, 0.0]
    kw = dict(scheme="ms", precision="fp32", green="fd", tol=0.0, max_iter=3, check_every=1)
    with L.Grid(mask) as g:
        L.lsfft_debug_inject(g.handle, 1)
        with pytest.raises(L.LsfftError) as ei:
            g.solve(10.0, e, **kw)
        assert ei.value.status == L.ECUDA
        assert "bounded wait" in str(ei.value)
        L.lsfft_debug_inject(g.handle, 0)
        r = g.solve(10.0, e, **kw)
        assert r.status == L.ENOTCONV
        ref = S.solve(S.Problem(mask, 10.0, np.array(e), "fd"), "ms", tol=0.0, max_iter=3)
        assert np.max(np.abs(r.hist_sigma - ref.hist_sigma) / np.abs(ref.hist_sigma)) < 1e-5
    with pytest.raises(L.LsfftError):
        L.lsfft_debug_inject(0, 1)

"""Batched solves (concurrent grids, jobs in order per grid) against single solves."""
import numpy as np
import pytest

from synth import complex_sigma_ray, random_mask, rsa_disk_mask, square_array_mask

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


def test_batch_matches_single_solves_and_reports_bad_jobs(L):
    masks = [square_array_mask(64), rsa_disk_mask(128, seed=3)[0], random_mask((32, 128), 0.3, seed=9),
             square_array_mask(16, d=3)]
    grids = [L.Grid(m) for m in masks]
    sig = [10.0, 0.1, 3.0 + 4.0j, 0.5 + 0.2j]
    jobs = []
    for gi, g in enumerate(grids):
        e = [1.0, 0.0] if g.d == 2 else [1.0, 0.0, 0.0]
        for k, s1 in enumerate(sig):
            scheme = ("ms", "em", "ms_sub", "em_sub")[(gi + k) % 4]
            kw = dict(scheme=scheme, precision="fp32" if k % 2 == 0 else "fp64", green="fd", tol=1e-7, max_iter=300,
                      alpha=0.05, beta=20.0)
            jobs.append((g, s1, e, kw))
    jobs.insert(3, (grids[0], 0.0, [1.0, 0.0], dict(scheme="em")))   # EM undefined at sigma_1 = 0
    out = L.solve_batch(jobs)
    assert isinstance(out[3], L.LsfftError) and out[3].status == L.EINVAL
    for (g, s1, e, kw), r in zip(jobs, out):
        if isinstance(r, L.LsfftError):
            continue
        ref = g.solve(s1, e, **kw)
        assert r.status == ref.status and r.iterations == ref.iterations
        np.testing.assert_array_equal(r.hist_sigma, ref.hist_sigma)
        np.testing.assert_array_equal(r.field_numpy(), ref.field_numpy())
    for g in grids:
        g.close()


def test_batch_complex_sigma_sweep_over_uneven_microstructures(L):
    """A small version of the sweep: complex sigma_1 on a ray over RSA-disk
    microstructures of different sizes, accelerated scheme with per-microstructure
    Lanczos estimates of [alpha, beta]."""
    sizes = (128, 256, 128, 256)
    grids = [L.Grid(rsa_disk_mask(n, seed=s)[0]) for s, n in enumerate(sizes)]
    sig = complex_sigma_ray(count=32, seed=1000)
    jobs = []
    for g in grids:
        a, b, _, _ = g.lanczos_hull([1.0, 0.0], green="fd", precision="fp32", steps=40, cutoff=1e-6)
        assert 0 < a < b
        a, b = 0.95 * a, 1.05 * b
        for s1 in sig:
            # EM in H'' only where it is stable against rounding, else plain EM
            rate, limit = L.lsfft_substitution_rates(s1, a, b)
            scheme = "em_sub" if rate < 0.98 * limit else "em"
            jobs.append((g, s1, [1.0, 0.0], dict(scheme=scheme, green="fd", tol=1e-6, max_iter=1500, alpha=a,
                                                 beta=b)))
    assert any(j[3]["scheme"] == "em" for j in jobs) and any(j[3]["scheme"] == "em_sub" for j in jobs)
    out = L.solve_batch(jobs)
    for r in out:
        assert not isinstance(r, L.LsfftError)
        assert r.status == L.OK, (r.sigma1 if hasattr(r, "sigma1") else None, r.status)
        assert np.isfinite(r.sigma_star)
    for g in grids:
        g.close()

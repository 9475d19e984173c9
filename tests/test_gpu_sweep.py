"""The persistent batch executor (lsfft_solve_sweep): many solves on grids of
uneven sizes in one kernel launch.  Iterate by iterate against the FP64 oracle
for complex sigma_1 on random-sequential-addition disk masks, against the
single-grid path, status and rejection rules, and a larger mixed batch."""
import numpy as np
import pytest

from oracle import schemes as S
from synth import complex_sigma_ray, rsa_disk_mask, square_array_mask

pytestmark = pytest.mark.gpu

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


def test_sweep_matches_oracle_iterate_by_iterate(L):
    """Complex sigma_1 from the r e^(i theta) ray on 128^2 and 256^2 disk packings,
    all four schemes, both Green symbols, in one launch; a fixed iteration count so
    that every iterate is compared."""
    masks = [rsa_disk_mask(128, seed=3)[0], rsa_disk_mask(256, seed=9)[0]]
    sig = complex_sigma_ray(count=8, seed=1000)
    ab = (0.12, 7.5)
    grids = [L.Grid(m) for m in masks]
    jobs, refs = [], []
    plan = [("em_sub", "fd"), ("em", "fd"), ("ms", "trig"), ("ms_sub", "trig")]
    for gi, (g, m) in enumerate(zip(grids, masks)):
        for k, (sch, green) in enumerate(plan):
            s1 = sig[4 * gi + k]
            e = [0.8, 0.6]
            kw = dict(scheme=sch, precision="fp32", green=green, tol=0.0, max_iter=8, alpha=ab[0], beta=ab[1])
            jobs.append((g, s1, e, kw))
            refs.append(S.solve(S.Problem(m, s1, np.array(e), green), sch, alpha=ab[0], beta=ab[1], tol=0.0,
                                max_iter=8))
    out = L.solve_sweep(jobs)
    for r, ref, (g, s1, e, kw) in zip(out, refs, jobs):
        assert not isinstance(r, Exception), r
        assert r.iterations == 8 and r.status == L.ENOTCONV
        es = np.max(np.abs(r.hist_sigma - ref.hist_sigma) / np.abs(ref.hist_sigma))
        E = r.field_numpy()
        ee = np.linalg.norm(E - ref.E) / np.linalg.norm(ref.E)
        assert es < ST and ee < ET, (kw["scheme"], s1, es, ee)
        r.free()
    for g in grids:
        g.close()


def test_sweep_stop_rule_matches_single_solves(L):
    """With a stop rule, every job reports what the single-grid path reports for the
    same problem: status, iteration count (within one, FP32 rounding near the
    threshold) and sigma_*."""
    sizes = [128, 256, 512, 1024]
    masks = [rsa_disk_mask(n, seed=20 + i)[0] for i, n in enumerate(sizes)]
    grids = [L.Grid(m) for m in masks]
    sig = complex_sigma_ray(count=8, seed=7)
    jobs = []
    for i, g in enumerate(grids):
        for s1, sch in ((sig[2 * i], "em"), (sig[2 * i + 1], "ms")):
            jobs.append((g, s1, [1.0, 0.0], dict(scheme=sch, precision="fp32", green="fd", tol=1e-5, max_iter=300)))
    out = L.solve_sweep(jobs)
    for r, (g, s1, e, kw) in zip(out, jobs):
        ref = g.solve(s1, e, **kw)
        assert r.status == ref.status
        assert abs(r.iterations - ref.iterations) <= 1, (r.iterations, ref.iterations)
        assert abs(r.sigma_star - ref.sigma_star) < 1e-5 * abs(ref.sigma_star)
        ref.free()
        r.free()
    for g in grids:
        g.close()


def test_sweep_rejects_ineligible_jobs(L):
    with L.Grid(square_array_mask(64)) as small, L.Grid(square_array_mask(128)) as g:
        for job in [(small, 2.0, [1.0, 0.0], dict(precision="fp32")),   # 64 points: below the range
                    (g, 2.0, [1.0, 0.0], dict(precision="fp64"))]:       # FP64 fields
            with pytest.raises(L.LsfftError) as ei:
                L.solve_sweep([job])
            assert ei.value.status == L.EINVAL


def test_sweep_large_mixed_batch(L):
    """32 disk packings of 128^2 to 1024^2 (the sweep workload's shape) with two
    complex sigma_1 each: every job ends with a status and finite sigma_*, and a
    sample agrees with its single-grid solve."""
    sizes = [128] * 8 + [256] * 8 + [512] * 8 + [1024] * 8
    grids, hulls = [], []
    for s, n in enumerate(sizes):
        m, _ = rsa_disk_mask(n, seed=s)
        grids.append(L.Grid(m))
    sig = complex_sigma_ray(count=64, seed=1000)
    jobs = []
    for i, g in enumerate(grids):
        for k in range(2):
            jobs.append((g, sig[2 * i + k], [1.0, 0.0], dict(scheme="em", precision="fp32", green="fd", tol=1e-6,
                                                           max_iter=400)))
    out = L.solve_sweep(jobs)
    assert all(not isinstance(r, Exception) for r in out)
    assert all(r.status in (L.OK, L.ENOTCONV, L.EDIVERGED) for r in out)
    assert all(np.isfinite(r.sigma_star) for r in out if r.status != L.EDIVERGED)
    for idx in (0, 17, 40, 63):
        g, s1, e, kw = jobs[idx]
        ref = g.solve(s1, e, **kw)
        assert abs(out[idx].sigma_star - ref.sigma_star) < 1e-5 * abs(ref.sigma_star)
        ref.free()
    for r in out:
        r.free()
    for g in grids:
        g.close()

"""The allocation-free volume-average entry point, checked against the averages
lsfft_solve reports for its own field.

Some callers cannot allocate device memory (they must not block, or their
memory belongs to another allocator); lsfft_field_averages_noalloc serves them
with a static scratch array.  This file is collected last so that a run which
stops at the first failure has already run every other test."""
import numpy as np
import pytest

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


CASES = [((64, 128), 10.0, "fp32"), ((64, 128), 3.0 + 4.0j, "fp32"), ((64, 128), 10.0, "fp64"),
         ((16, 32, 16), 5.0 - 2.0j, "fp32"), ((1024, 512), 0.1, "fp32")]


@pytest.mark.parametrize("shape,s1,prec", CASES)
def test_noalloc_averages_match_solve(L, shape, s1, prec):
    import torch

    d = len(shape)
    mask = random_mask(shape, 0.3, seed=sum(shape))
    e = [0.6, 0.8] if d == 2 else [0.0, 0.6, 0.8]
    with L.Grid(mask) as g:
        # Moulinec-Suquet reports J = sigma E at every iterate, the quantity averaged here
        r = g.solve(s1, e, scheme="ms", precision=prec, green="fd", tol=0.0, max_iter=6)
        ref = np.concatenate([[m.real, m.imag, j.real, j.imag] for m, j in zip(r.mean_E, r.mean_J)])
        ref_sig = r.sigma_star
        mask_dev = torch.from_numpy(mask).cuda()
        torch.cuda.synchronize()
        outs = []
        for _ in range(2):                                   # two calls in a row share the scratch array
            out = torch.full((4 * d + 3,), float("nan"), dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            L.lsfft_field_averages_noalloc(d, tuple(reversed(shape)), r._ptr.contents.E_device,
                                           L.FP32 if prec == "fp32" else L.FP64, mask_dev.data_ptr(), s1, e,
                                           out.data_ptr(), 0)
            torch.cuda.synchronize()
            outs.append(out.cpu().numpy())
        r.free()
    tol = 1e-5 if prec == "fp32" else 1e-12
    for o in outs:
        got = o[:4 * d]
        assert np.all(np.abs(got - ref) <= tol * np.abs(ref).max())
        sig = complex(o[4 * d + 1], o[4 * d + 2])
        assert abs(sig - ref_sig) <= tol * abs(ref_sig)
    np.testing.assert_array_equal(outs[0], outs[1])


def test_noalloc_rejects_bad_arguments(L):
    import torch

    out = torch.zeros(16, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(L.LsfftError) as ei:                  # beyond the scratch limit: 2^28 + voxels
        L.lsfft_field_averages_noalloc(2, (32768, 16385), dummy.data_ptr(), L.FP32, dummy.data_ptr(), 2.0,
                                       [1.0, 0.0], out.data_ptr(), 0)
    assert ei.value.status == L.EINVAL and "limit" in str(ei.value)
    with pytest.raises(L.LsfftError) as ei:
        L.lsfft_field_averages_noalloc(4, (16, 16, 16), dummy.data_ptr(), L.FP32, dummy.data_ptr(), 2.0,
                                       [1.0, 0.0, 0.0], out.data_ptr(), 0)
    assert ei.value.status == L.EINVAL

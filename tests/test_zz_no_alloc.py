"""The allocation-free volume-average entry point, checked against the averages
lsfft_solve reports for its own field and against plain numpy means of that
field copied to the host.

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


# the last three span many partial sums of 65536 voxels in FP32, FP64 and 3-D
CASES = [((64, 128), 10.0, "fp32"), ((64, 128), 3.0 + 4.0j, "fp32"), ((64, 128), 10.0, "fp64"),
         ((16, 32, 16), 5.0 - 2.0j, "fp32"), ((1024, 512), 0.1, "fp32"), ((512, 256), 2.0 - 1.0j, "fp64"),
         ((32, 64, 64), 7.0, "fp32")]


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
        # the same averages by plain numpy on the host copy of the field
        E = r.field_numpy().astype(np.complex128).reshape(d, -1)
        sig = np.where(mask.reshape(-1) != 0, complex(s1), 1.0)
        mE, mJ = E.mean(axis=1), (sig[None] * E).mean(axis=1)
        host = np.concatenate([[a.real, a.imag, b.real, b.imag] for a, b in zip(mE, mJ)])
        host_norm = float(np.mean(np.sum(np.abs(E) ** 2, axis=0)))
        host_sig = complex(np.dot(mJ, e) / np.dot(mE, e))
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
        # the field is read in the precision it is stored in, summed in FP64: against the
        # numpy means of the same values only the summation order differs
        assert np.all(np.abs(got - host) <= 1e-12 * np.abs(host).max())
        assert abs(o[4 * d] - host_norm) <= 1e-12 * host_norm
        assert abs(sig - host_sig) <= 1e-11 * abs(host_sig)
    np.testing.assert_array_equal(outs[0], outs[1])


def test_noalloc_accepts_the_largest_field(L):
    """Exactly 2^28 voxels (16384 x 16384), the most the scratch array holds: E = (1, 0)
    everywhere on a half-filled mask gives <E> = (1, 0), <J_x> = (sigma_1 + 1)/2,
    <|E|^2> = 1 and sigma_* = <J_x>, in closed form."""
    import torch

    n = 16384
    E = torch.zeros((2, n, n), dtype=torch.complex64, device="cuda")
    E[0] = 1.0
    mask = torch.zeros((n, n), dtype=torch.uint8, device="cuda")
    mask[: n // 2] = 1
    s1 = 3.0 - 1.0j
    for _ in range(2):
        out = torch.full((11,), float("nan"), dtype=torch.float64, device="cuda")
        L.lsfft_field_averages_noalloc(2, (n, n), E.data_ptr(), L.FP32, mask.data_ptr(), s1, [1.0, 0.0],
                                       out.data_ptr(), 0)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        jx = (s1 + 1.0) / 2.0
        np.testing.assert_allclose(o, [1, 0, jx.real, jx.imag, 0, 0, 0, 0, 1, jx.real, jx.imag], atol=1e-12)
    del E, mask
    torch.cuda.empty_cache()


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
    with pytest.raises(L.LsfftError) as ei:                  # a vanishing applied field
        L.lsfft_field_averages_noalloc(2, (4, 4), dummy.data_ptr(), L.FP32, dummy.data_ptr(), 2.0,
                                       [0.0, 0.0], out.data_ptr(), 0)
    assert ei.value.status == L.EINVAL

"""With MXFFT_OPT_FOLD_STATS the round trip on the tensor-core path takes the
inverse transform's Alg. 1 statistics inside the forward columns pass (every
stored value goes through the same accumulator as the statistics kernel; each
CTA flushes one segment per run of tiles of a slice).  The inverse exponent it selects must equal the
one the stand-alone statistics kernel selects on the same forward output, for
every slice, whatever the slices' scales and however the tiles of a slice are
split between CTAs; the round trip itself stays equal to the emulation and,
through the executor, to the plan call.

Inputs give every slice its own power-of-two scale (exponents from -40 to
+40), so that a record receiving another slice's values, or missing a CTA's
segment, selects a different exponent.  One slice is all zeros (k = 0).
"""
import os
import sys

import numpy as np
import pytest

from paper_2512_04317_gb300 import phantom
from parity_util import assert_close_to_emulation

sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
import tc16_ref  # noqa: E402

pytestmark = pytest.mark.gpu


def scaled_slices(batch, n0, n1, seed):
    x = phantom.random_complex((batch, n0, n1), seed=seed)
    rng = np.random.default_rng(seed)
    e = rng.integers(-40, 41, size=batch)
    x *= (2.0 ** e).astype(np.float32)[:, None, None]
    if batch > 2:
        x[batch // 2] = 0
    return x


def stats_kernel_exponents(y, fmt):
    import torch

    from paper_2512_04317_gb300 import mxfft
    batch = y.shape[0]
    k = torch.full((batch,), -9999, dtype=torch.int32, device=y.device)
    stream = torch.cuda.current_stream(y.device).cuda_stream
    st = mxfft.mxfft_prescale_exponents_noalloc(y.data_ptr(), batch, y.shape[-2], y.shape[-1], fmt,
                                                1e-3, 0.5, k.data_ptr(), stream)
    assert st == mxfft.MXFFT_OK, mxfft.status_string(st)
    torch.cuda.synchronize()
    return k.cpu().tolist()


# (n0, n1, batch): several slices per CTA (256 x 256: 16 tiles a slice), a
# slice's tiles split over two or three CTAs (512 x 512, 1024 x 1024), mixed
# lengths, and n0 = 2048 (columns tiles strided over the CTAs: the separate
# statistics pass, same exponents)
CASES = [(256, 256, 64), (256, 256, 301), (512, 512, 13), (512, 256, 37), (256, 1024, 21),
         (1024, 1024, 5), (1024, 512, 7), (2048, 256, 3)]


@pytest.mark.parametrize("n0,n1,batch", CASES)
@pytest.mark.parametrize("fmt", ["e4m3", "e5m2"])
def test_folded_inverse_exponents_equal_statistics_kernel(n0, n1, batch, fmt, cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = torch.from_numpy(scaled_slices(batch, n0, n1, seed=n0 + n1 + batch)).cuda()
    with mxfft.Plan(n0, n1, fmt, 32, path="tc16", fold_stats=True) as p:
        y = p.forward(x)
        torch.cuda.synchronize()
        _, flags_f, k_f = p.status()
        p.roundtrip(x)
        torch.cuda.synchronize()
        st, flags, k_rt = p.status()
    assert st == 0 and flags == 0 and flags_f == 0
    k_inv_kernel = stats_kernel_exponents(y, fmt)
    assert [kk[0] for kk in k_rt] == list(k_f)
    assert [kk[1] for kk in k_rt] == k_inv_kernel
    assert k_rt[batch // 2] == [0, 0] if batch > 2 else True


@pytest.mark.parametrize("n0,n1,batch", [(256, 256, 9), (512, 512, 3), (1024, 256, 4)])
def test_folded_round_trip_matches_emulation(n0, n1, batch, cuda_device):
    import torch

    from paper_2512_04317_gb300 import mxfft
    x = scaled_slices(batch, n0, n1, seed=7 * batch)
    xt = torch.from_numpy(x).cuda()
    with mxfft.Plan(n0, n1, "e4m3", 32, path="tc16", fold_stats=True) as p:
        got = p.roundtrip(xt).cpu().numpy()
        assert p.status()[1] == 0
    with mxfft.Plan(n0, n1, "e4m3", 32, path="tc16", fold_stats=False) as p:
        unfolded = p.roundtrip(xt).cpu().numpy()
    np.testing.assert_array_equal(got.view(np.uint32), unfolded.view(np.uint32))
    want = tc16_ref.mxfft2d(x, "e4m3", "roundtrip")
    assert_close_to_emulation(got, want, (n0, n1, batch))


def test_engine_folds_only_round_trip_slices(cuda_device):
    # one tensor-core plan with a forward item and a round-trip item in the
    # same columns launch: only the round trip's slices carry records for the
    # folded statistics; results and exponents equal the plan calls
    import torch

    from paper_2512_04317_gb300 import mxfft
    xa = torch.from_numpy(scaled_slices(5, 512, 512, seed=3)).cuda()
    xb = torch.from_numpy(scaled_slices(6, 512, 512, seed=4)).cuda()
    xc = torch.from_numpy(scaled_slices(3, 512, 512, seed=5)).cuda()
    with mxfft.Plan(512, 512, "e4m3", 32, path="tc16", fold_stats=False) as p:
        wa = p.forward(xa).cpu().numpy()
        wb = p.roundtrip(xb).cpu().numpy()
        kb = p.status()[2]
        wc = p.roundtrip(xc).cpu().numpy()
        kc = p.status()[2]
    for fold in (True, False):
        with mxfft.Engine(tc16=True, graphs=True, fold_stats=fold) as eng:
            ya, yb, yc = torch.empty_like(xa), torch.empty_like(xb), torch.empty_like(xc)
            eng.run([("forward", xa, ya, "e4m3", 32), ("roundtrip", xb, yb, "e4m3", 32),
                     ("roundtrip", xc, yc, "e4m3", 32)])
            torch.cuda.synchronize()
            flags, k = eng.status()
            launches = eng.launches_per_run()
        assert flags == 0
        for got, want in ((ya, wa), (yb, wb), (yc, wc)):
            np.testing.assert_array_equal(got.cpu().numpy().view(np.uint32), want.view(np.uint32))
        assert [kk[1] for kk in k[5:11]] == [kk[1] for kk in kb]
        assert [kk[1] for kk in k[11:]] == [kk[1] for kk in kc]
        # statistics, rows, columns, (statistics of the forward outputs,)
        # inverse rows, inverse columns
        assert launches == (5 if fold else 6)

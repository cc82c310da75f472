"""GPU parity of HEALPix-SSIM and the L1 + HSSIM loss (Sec. 4.1) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_29794_b300 import raster as R
from paper_2606_29794_b300 import synth as S
from tests.gpu_util import mask_from_words

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]


def _mask_words(view):
    import ctypes
    from paper_2606_29794_b300 import _lib as L
    k = view["nside_log2"]
    words = torch.empty(12 * 4 ** k // 32, dtype=torch.int32, device="cuda")
    rast = R.Rasterizer()
    L.check(L.lib().hpxgs_mask_build(L.make_views([view]), ctypes.byref(rast.cfg), ctypes.c_void_p(words.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)), "mask")
    return words


@pytest.mark.parametrize("k,kind,fov,lam", [(5, 0, 360.0, 0.2), (6, 2, 190.0, 0.2), (7, 1, 90.0, 0.5), (4, 2, 220.0, 1.0)])
def test_hssim_loss_and_grad(k, kind, fov, lam):
    rng = np.random.default_rng(k)
    n = 12 * 4 ** k
    I = rng.random((n, 3)).astype(np.float32)
    G = np.clip(I + rng.normal(0, 0.1, (n, 3)), 0, 1).astype(np.float32)
    view = S.make_view(k, kind, fov)
    words = _mask_words(view)
    It = torch.tensor(I, device="cuda", requires_grad=True)
    Gt = torch.tensor(G, device="cuda")
    loss, parts = R.hssim_loss(It, Gt, words, k, lam)
    loss.backward()
    torch.cuda.synchronize()
    m = mask_from_words(words.cpu().numpy().view(np.uint32), n)
    ref_loss, ref_h, ref_l1, ref_dI = O.hssim_loss(2 ** k, I.astype(np.float64), G.astype(np.float64), m, lam)
    assert abs(parts[1].item() - ref_h) < 2e-6
    assert abs(parts[2].item() - ref_l1) < 2e-6
    assert abs(loss.item() - ref_loss) < 2e-6
    g = It.grad.cpu().numpy().astype(np.float64)
    assert np.abs(g - ref_dI).max() <= 1e-3 * np.abs(ref_dI).max()
    assert np.linalg.norm(g - ref_dI) <= 1e-3 * np.linalg.norm(ref_dI)


def test_hssim_identical_maps_is_one():
    k = 6
    n = 12 * 4 ** k
    I = torch.rand((n, 3), device="cuda")
    words = _mask_words(S.make_view(k))
    loss, parts = R.hssim_loss(I, I.clone(), words, k, 0.2)
    assert abs(parts[1].item() - 1.0) < 1e-6 and abs(loss.item()) < 1e-6


@pytest.mark.parametrize("k,kind,fov", [(5, 0, 360.0), (6, 2, 190.0), (7, 1, 90.0), (9, 2, 190.0)])
def test_window_table_path_is_bit_identical(k, kind, fov):
    import ctypes
    from paper_2606_29794_b300 import _lib as L
    rng = np.random.default_rng(k + 100)
    n = 12 * 4 ** k
    I = torch.tensor(rng.random((n, 3)), dtype=torch.float32, device="cuda")
    G = torch.tensor(rng.random((n, 3)), dtype=torch.float32, device="cuda")
    words = _mask_words(S.make_view(k, kind, fov))
    tab = R.hssim_table(words, k)
    nb = ctypes.c_size_t()
    L.check(L.lib().hpxgs_hssim_workspace_size(k, ctypes.byref(nb)), "ws")
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    outs = []
    for use_table in (False, True):
        ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
        out3 = torch.empty(3, device="cuda")
        dI = torch.empty((n, 3), device="cuda")
        if use_table:
            L.check(L.lib().hpxgs_hssim_forward_table(p(I), p(G), p(words), k, 0.2, p(tab), p(ws), nb.value, p(out3), s), "f")
            L.check(L.lib().hpxgs_hssim_backward_table(p(I), p(G), p(words), k, 0.2, p(tab), p(ws), nb.value, None, p(dI), s), "b")
        else:
            L.check(L.lib().hpxgs_hssim_forward(p(I), p(G), p(words), k, 0.2, p(ws), nb.value, p(out3), s), "f")
            L.check(L.lib().hpxgs_hssim_backward(p(I), p(G), p(words), k, 0.2, p(ws), nb.value, None, p(dI), s), "b")
        torch.cuda.synchronize()
        outs.append((out3.clone(), dI.clone()))
    assert torch.equal(outs[0][0], outs[1][0])
    assert torch.equal(outs[0][1], outs[1][1])

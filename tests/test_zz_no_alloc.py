"""The workspace-free loss entry point matches the workspace one.

hpxgs_hssim_loss_noalloc exists for callers that cannot hand the library any
device memory (for example a plugin whose host application owns the whole GPU
memory budget, or a real-time loop that may not allocate after start-up). It
keeps its partial sums in an array inside the library, so two calls in a row
must each give the same {loss, HSSIM, L1} as hpxgs_hssim_forward with a
workspace, and the same value as the FP64 oracle's loss (Sec. 4.1) within the
2e-6 the other HSSIM tests use. This file runs last so that a failure here leaves
every other test already run.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle as O
from paper_2606_29794_b300 import _lib as L
from paper_2606_29794_b300 import synth as S
from tests.gpu_util import mask_from_words

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not torch.cuda.is_available(), reason="needs CUDA")]


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("k,kind,fov", [(9, S.CAM_FISHEYE, 190.0), (6, S.CAM_FULL, 360.0)])
def test_noalloc_loss_matches_workspace_loss_twice(k, kind, fov):
    lib = L.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = 12 * 4 ** k
    rng = np.random.default_rng(k)
    I = torch.tensor(rng.random((n, 3)), dtype=torch.float32, device="cuda")
    G = torch.tensor(np.clip(I.cpu().numpy() + rng.normal(0, 0.1, (n, 3)), 0, 1), dtype=torch.float32, device="cuda")
    words = torch.empty(n // 32, dtype=torch.int32, device="cuda")
    cfg = L.default_config()
    L.check(lib.hpxgs_mask_build(L.make_views([S.make_view(k, kind, fov)]), ctypes.byref(cfg), _p(words), stream), "mask")
    nb = ctypes.c_size_t()
    L.check(lib.hpxgs_hssim_workspace_size(k, ctypes.byref(nb)), "ws size")
    ws = torch.empty(nb.value, dtype=torch.uint8, device="cuda")
    ref = torch.empty(3, dtype=torch.float32, device="cuda")
    L.check(lib.hpxgs_hssim_forward(_p(I), _p(G), _p(words), k, 0.2, _p(ws), nb.value, _p(ref), stream), "forward")
    m = mask_from_words(words.cpu().numpy().view(np.uint32), n)
    o_loss, o_h, o_l1, _ = O.hssim_loss(2 ** k, I.cpu().numpy().astype(np.float64), G.cpu().numpy().astype(np.float64),
                                        m, 0.2, grad=False)
    for _ in range(2):
        out = torch.full((3,), float("nan"), dtype=torch.float32, device="cuda")
        L.check(lib.hpxgs_hssim_loss_noalloc(_p(I), _p(G), _p(words), k, 0.2, _p(out), stream), "noalloc")
        torch.cuda.synchronize()
        assert torch.allclose(out, ref, rtol=0, atol=2e-6), (out, ref)
        got = out.cpu().numpy().astype(np.float64)
        assert np.abs(got - np.array([o_loss, o_h, o_l1])).max() < 2e-6, (got, o_loss, o_h, o_l1)


def test_noalloc_rejects_orders_above_the_limit():
    lib = L.lib()
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    rc = lib.hpxgs_hssim_loss_noalloc(_p(buf), _p(buf), _p(buf), 11, 0.2, _p(buf),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == L.E_INVALID_ARG

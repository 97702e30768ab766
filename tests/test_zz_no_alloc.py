"""gmr_l2_loss_noalloc, the loss entry point that allocates nothing (for
callers that must not call cudaMalloc where they compute the loss: a
latency-critical loop in which an allocation could synchronise the device,
or a process whose device memory belongs to its own pool). Called through
the C ABI and compared with gmr_l2_loss, which uses a context's workspace,
on two calls in a row; the second call is smaller than the first, so it
runs over partial sums left in the library's scratch array by the first."""

import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_loss_matches_context_loss_on_two_calls():
    from paper_2602_14493_b300 import Renderer, _lib

    L = _lib.load()
    r = Renderer()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for seed, n in ((1, 3 * 1024 * 1024 + 7), (2, 3 * 301 * 257 + 5)):
        g = torch.Generator(device="cuda").manual_seed(seed)
        img = torch.rand(n, device="cuda", generator=g)
        tgt = torch.rand(n, device="cuda", generator=g)
        ref_loss, ref_grad = r.l2_loss(img, tgt)
        grad = torch.full_like(img, float("nan"))
        loss = torch.full((), float("nan"), dtype=torch.float64, device="cuda")
        st = L.gmr_l2_loss_noalloc(_p(img), _p(tgt), n, _p(grad), _p(loss), stream)
        assert st == _lib.GMR_OK
        torch.cuda.synchronize()
        assert torch.equal(grad, ref_grad)
        assert abs(float(loss) - float(ref_loss)) <= 1e-12 * abs(float(ref_loss))
        expect = float(((img.double() - tgt.double()) ** 2).sum())
        assert abs(float(loss) - expect) <= 1e-6 * expect
    # sizes beyond the entry point's stated maximum (GMR_L2_NOALLOC_MAX_ELEMS)
    # are rejected before anything runs
    st = L.gmr_l2_loss_noalloc(_p(img), _p(tgt), _lib.GMR_L2_NOALLOC_MAX_ELEMS + 1, _p(grad), _p(loss), stream)
    assert st == 4  # GMR_ERR_CAPACITY
    assert L.gmr_l2_loss_noalloc(_p(img), _p(tgt), -1, _p(grad), _p(loss), stream) == 1
    r.close()

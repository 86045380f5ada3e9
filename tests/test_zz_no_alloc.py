"""ug_mse_loss_grad_static, the entry point for callers that cannot allocate
device memory (for example code running inside a stream capture, or a plugin
that is only handed the buffers it works on): its partial sums live in the
library's own static device array. Checked through the C ABI against
ug_mse_loss_grad on two calls in a row. Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2505_05643_gb300 import binding as B

pytestmark = pytest.mark.gpu


def _reference(img, tgt, n):
    grad = torch.empty_like(img)
    loss = torch.empty(B.UG_MSE_LOSS_FLOATS, device="cuda")
    B.ug_mse_loss_grad(img, tgt, n, grad, loss)
    return grad, loss[:1]


def test_static_scratch_matches_allocating_entry_point_twice():
    lib = B.load()
    rng = np.random.default_rng(77)
    # two calls in a row, the second smaller than the first: nothing of the
    # first call's scratch may leak into the second
    for n in (3 * 65536 + 123, 1000):
        img = torch.from_numpy(rng.uniform(0, 1, n).astype(np.float32)).cuda()
        tgt = torch.from_numpy(rng.uniform(0, 1, n).astype(np.float32)).cuda()
        grad = torch.full_like(img, float("nan"))
        loss = torch.full((1,), float("nan"), device="cuda")
        st = lib.ug_mse_loss_grad_static(img.data_ptr(), tgt.data_ptr(), n, grad.data_ptr(),
                                         loss.data_ptr(), torch.cuda.current_stream().cuda_stream)
        assert st == B.UG_OK
        g_ref, l_ref = _reference(img, tgt, n)
        torch.cuda.synchronize()
        # the gradient is the same elementwise formula; the loss sums in another order
        torch.testing.assert_close(grad, g_ref, rtol=0, atol=0)
        np.testing.assert_allclose(loss.item(), l_ref.item(), rtol=1e-6)
        d = img.double() - tgt.double()
        np.testing.assert_allclose(loss.item(), float((d * d).mean()), rtol=1e-6)


def test_static_scratch_rejects_sizes_beyond_its_limit():
    lib = B.load()
    small = torch.zeros(4, device="cuda")
    st = lib.ug_mse_loss_grad_static(small.data_ptr(), small.data_ptr(),
                                     B.UG_MSE_STATIC_MAX_N + 1, None, small.data_ptr(), None)
    assert st == B.UG_ERR_INVALID_ARGUMENT
    st = lib.ug_mse_loss_grad_static(small.data_ptr(), small.data_ptr(), 0, None,
                                     small.data_ptr(), None)
    assert st == B.UG_ERR_INVALID_ARGUMENT

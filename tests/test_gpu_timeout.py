"""The bounded device-side waits of the tensor-core kernels: a forward whose
tile waits are set to give up at once reports STDA_ERR_TIMEOUT through
stda_device_status (the kernels finish the MMAs they issued, free their
tensor memory and return), and the same context then runs a normal forward
that matches the FP64 oracle. No GPU fault or hang is involved: the limit
is a poll count, the waits for issued MMAs keep their default bound."""
import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def stda():
    from paper_2307_09063_gb300 import build

    build.build()
    from paper_2307_09063_gb300 import stda as S

    return S


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_wait_timeout_is_reported_and_context_recovers(stda, weights, prec):
    rng = np.random.default_rng(99)
    x = torch.from_numpy(rng.uniform(0, 1, (2, 3, 64, 64)).astype(np.float32)).to(torch.bfloat16)
    xd = x.cuda()
    ctx = stda.Context(64, 64, 2, prec, 0)
    assert ctx.device_status() == stda.OK
    ctx.set_wait_limit(0)
    ctx.forward(xd)
    assert ctx.device_status() == stda.ERR_TIMEOUT
    assert ctx.device_status() == stda.OK  # the read cleared the word
    ctx.set_wait_limit()
    got = ctx.forward(xd)[:, 0].float().cpu().numpy()
    assert ctx.device_status() == stda.OK
    ref = O.forward_batch(*weights, x.float().numpy())
    assert np.max(np.abs(got - ref)) <= 2e-2

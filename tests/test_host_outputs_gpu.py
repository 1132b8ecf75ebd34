"""Per-event outputs in pinned host memory: the kernels store into host
memory directly (mapped pinned memory, NVLink-C2C on Grace-Blackwell), with
results identical to device-resident outputs; pageable host memory is
rejected with an error code."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_1002_3446_gb300 as tess  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    c = tess.tess_init(0)
    yield c
    tess.tess_destroy(c)


@pytest.mark.parametrize("n,precision,N", [(6, tess.TESS_FP32_DS, 700_001), (10, tess.TESS_FP32_DS, 200_003),
                                           (5, tess.TESS_FP64, 100_000)])
def test_host_outputs_equal_device_outputs(ctx, n, precision, N):
    p = tess.process(n, precision=precision, pt_min=30.0 if n >= 10 else 20.0, hist_bins=20,
                     hist_observable=tess.TESS_OBS_PTLEAD, hist_lo=20.0, hist_hi=400.0)
    dev = tess.Run(ctx, p, N)
    host = tess.Run(ctx, p, N, host_per_event=True)
    assert not host.t["weight"].is_cuda and host.t["weight"].is_pinned()
    dev.generate(4, 1 << 30)
    host.generate(4, 1 << 30)
    torch.cuda.synchronize()
    for key in ("weight", "me2", "pass", "ht", "ptlead", "rmin"):
        assert np.array_equal(dev.t[key].cpu().numpy(), host.t[key].numpy()), key
    assert np.array_equal(dev.acc.cpu().numpy(), host.acc.cpu().numpy())
    assert np.array_equal(dev.hist.cpu().numpy(), host.hist.cpu().numpy())


def test_pageable_host_output_rejected(ctx):
    p = tess.process(6)
    run = tess.Run(ctx, p, 1000)
    pageable = torch.empty(1000, dtype=torch.float64)
    outs = tess.make_outputs(pageable, None, None, None, None, None, run.acc, None)
    with pytest.raises(tess.TessError) as e:
        tess.tess_generate(ctx, p, 1, 0, 1000, outs, run.workspace)
    assert e.value.code == tess.TESS_E_INVALID
    assert "weight" in tess.tess_last_error()

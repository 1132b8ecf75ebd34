"""The allocation-free entry point, tess_generate_noalloc.

It exists for callers that cannot allocate device memory or give the library
a workspace (a host program whose memory manager owns the whole device, a
latency-critical loop that cannot take an allocation's implicit
synchronisation); its scratch is a fixed array inside the library.  Here it is
called through the C ABI twice in a row -- the second call finds the first
call's leftovers in that shared array -- and each call's outputs are compared
with tess_generate's for the same events, at the FP64 parity tolerance the
other tests use (relative 1e-10); the FP32 exact-sum case runs the same
fused kernel as tess_generate and must agree bit for bit.  Sampled events at
the FP32 precisions need tess_generate's workspace and are refused.  This file is collected last so that a run
stopping at the first failure has run every other test already; it also
passes on its own in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

import paper_1002_3446_gb300 as tess  # noqa: E402

RTOL = 1e-10


def _close(a, b):
    a, b = np.asarray(a), np.asarray(b)
    scale = np.maximum(np.abs(b), 1e-300)
    return np.all((np.abs(a - b) <= RTOL * scale) | (a == b))


def _outputs_of(run):
    torch.cuda.synchronize()
    d = {k: v.cpu().numpy() for k, v in run.t.items() if v is not None}
    d["acc"] = run.acc.cpu().numpy()
    d["hist"] = run.hist.cpu().numpy() if run.hist is not None else None
    return d


@pytest.fixture(scope="module")
def ctx():
    assert torch.cuda.is_available()
    c = tess.tess_init(0)
    yield c
    tess.tess_destroy(c)


CALLS = [
    # (process, seed, first event, events)
    (dict(n=6, precision=tess.TESS_FP64, hist_bins=40, hist_observable=tess.TESS_OBS_HT, hist_lo=200.0,
          hist_hi=3000.0), 1, 0, 5000),
    (dict(n=4, precision=tess.TESS_FP64, helicity_mode=tess.TESS_HEL_SUM, hist_bins=50), 2, 12345, 3001),
]

CALLS_FP32 = [
    (dict(n=4, precision=tess.TESS_FP32_CURRENTS, helicity_mode=tess.TESS_HEL_SUM, hist_bins=50), 3, 777, 2049),
    (dict(n=5, precision=tess.TESS_FP32_DS, helicity_mode=tess.TESS_HEL_SUM), 4, 0, 1000),
]


def test_noalloc_matches_generate_on_two_calls_in_a_row(ctx):
    for kw, seed, first, N in CALLS:
        proc = tess.process(**kw)
        ref = tess.Run(ctx, proc, N)
        ref.generate(seed, first)
        got = tess.Run(ctx, proc, N)  # the test owns the outputs; the entry point allocates nothing
        tess.tess_generate_noalloc(ctx, proc, seed, first, N, got.outputs)
        a, b = _outputs_of(got), _outputs_of(ref)
        assert np.array_equal(a["pass"], b["pass"])
        for key in ("weight", "me2", "ht", "ptlead", "rmin"):
            assert _close(a[key], b[key]), key
        sa, sb = got.result(), ref.result()
        assert abs(sa[0] - sb[0]) <= RTOL * abs(sb[0]) and sa[2:] == sb[2:]
        ha, _ = got.histograms()
        hb, _ = ref.histograms()
        assert np.allclose(ha, hb, rtol=RTOL, atol=1e-12 * hb.sum())


def test_noalloc_fp32_exact_sum_matches_generate(ctx):
    for kw, seed, first, N in CALLS_FP32:
        proc = tess.process(**kw)
        ref = tess.Run(ctx, proc, N)
        ref.generate(seed, first)
        got = tess.Run(ctx, proc, N)
        for _ in range(2):
            got.reset()
            tess.tess_generate_noalloc(ctx, proc, seed, first, N, got.outputs)
            a, b = _outputs_of(got), _outputs_of(ref)
            for key in ("pass", "weight", "me2", "ht", "ptlead", "rmin"):
                assert np.array_equal(a[key], b[key]), key
            sa, sb = got.result(), ref.result()
            assert abs(sa[0] - sb[0]) <= RTOL * abs(sb[0]) and sa[2:] == sb[2:]


def test_noalloc_refuses_fp32_sampled(ctx):
    for prec in (tess.TESS_FP32_CURRENTS, tess.TESS_FP32_DS):
        proc = tess.process(6, precision=prec)
        run = tess.Run(ctx, proc, 16)
        with pytest.raises(tess.TessError) as e:
            tess.tess_generate_noalloc(ctx, proc, 1, 0, 16, run.outputs)
        assert e.value.code == tess.TESS_E_UNSUPPORTED
        assert "TESS_FP64 only" in tess.tess_last_error()


def test_noalloc_host_mapped_outputs(ctx):
    # per-event arrays in pinned host memory, stored by the kernel directly
    proc = tess.process(6, precision=tess.TESS_FP64)
    N = 1000
    ref = tess.Run(ctx, proc, N)
    tess.tess_generate_noalloc(ctx, proc, 5, 100, N, ref.outputs)
    got = tess.Run(ctx, proc, N, host_per_event=True)
    tess.tess_generate_noalloc(ctx, proc, 5, 100, N, got.outputs)
    a, b = _outputs_of(got), _outputs_of(ref)
    for key in ("pass", "weight", "me2", "ht", "ptlead", "rmin"):
        assert np.array_equal(a[key], b[key]), key


def test_noalloc_rejects_too_many_bins(ctx):
    proc = tess.process(6, hist_bins=tess.TESS_NOALLOC_MAX_BINS + 1)
    run = tess.Run(ctx, proc, 16)
    with pytest.raises(tess.TessError) as e:
        tess.tess_generate_noalloc(ctx, proc, 1, 0, 16, run.outputs)
    assert e.value.code == tess.TESS_E_INVALID
    assert "histogram bins" in tess.tess_last_error()

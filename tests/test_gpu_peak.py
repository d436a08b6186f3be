"""The FP32 throughput probe does the arithmetic it reports.

Every chain runs x <- a x + b with a = 1 - 2^-20, b = 2^-20, whose closed
form after n steps is x_n = 1 + (x_0 - 1) a^n; each thread writes the sum of
its 8 chains (16 values in the packed form). The probe must report
2 flops per fused multiply-add over every thread, chain and step.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nb():
    from paper_2405_01420_gb300 import nb as nbmod
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    nbmod.load_library()
    return nbmod


@pytest.mark.parametrize("packed", [False, True])
def test_probe_chains_follow_their_closed_form(nb, packed):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks_per_sm, iters = 2, 64
    threads = sms * blocks_per_sm * 256
    out = torch.full((threads,), float("nan"), dtype=torch.float32, device="cuda")
    flops = nb.nb_fp32_peak_probe(out, packed=packed, blocks_per_sm=blocks_per_sm, iters=iters)
    torch.cuda.synchronize()
    steps = iters * 16
    assert flops == 2.0 * (2 if packed else 1) * threads * steps * 8
    a = 1.0 - 2.0 ** -20
    an = a ** steps
    tid = np.arange(threads)
    c = np.arange(8)
    x0 = 1e-3 * (tid[:, None] & 255).astype(np.float64) + c[None, :]
    want = (1.0 + (x0 - 1.0) * an).sum(1)
    if packed:
        want = want + (1.0 + (0.5 * c[None, :] - 1.0) * an).sum(1)
    got = out.cpu().numpy().astype(np.float64)
    # every chain value stays below 8, so each step rounds by at most half an ulp of 8 (2^-21):
    # at most steps * 2^-21 per chain, 16 chain values per thread; a run of half the steps would
    # be off by about 3e-2
    np.testing.assert_allclose(got, want, rtol=0, atol=16 * steps * 2.0 ** -21 + 1e-5)


def test_probe_rejects_a_short_output(nb):
    out = torch.empty(16, dtype=torch.float32, device="cuda")
    with pytest.raises(nb.NBError):
        nb.nb_fp32_peak_probe(out, blocks_per_sm=1, iters=1)

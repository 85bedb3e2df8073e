"""mfs_fp32_fma_rate: the FP32 FMA throughput the pair kernel's roofline divides by, measured on the
device.  It must land near 2 x 128 lanes x SMs x SM clock (the FMA pipe's rate), for the packed
f32x2 form the Stokeslet kernel issues and for scalar fma."""

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__

    __graft_entry__.build()


@pytest.mark.parametrize("packed", [True, False])
def test_fma_rate_near_the_pipe_rate(packed):
    from paper_2409_04215_gb300.api import fp32_fma_rate

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = 2 * 128 * sms * 2.07e9 / 1e12  # at the maximum SM clock
    rate = fp32_fma_rate(packed)
    # a lower SM clock under another tenant's load or a power cap lowers it; more than the nominal
    # rate would mean the chains were not executed
    assert 0.4 * nominal < rate < 1.02 * nominal, (rate, nominal)


@pytest.mark.parametrize("mode", [2, 3, 4])
def test_fma_rate_operand_patterns(mode):
    """The probe's other operand patterns (distinct, rewritten operand registers; the Stokeslet
    kernel's 8 warps per SM) time real work: below the nominal rate, above a fifth of it."""
    from paper_2409_04215_gb300.api import fp32_fma_rate

    sms = torch.cuda.get_device_properties(0).multi_processor_count
    nominal = 2 * 128 * sms * 2.07e9 / 1e12
    rate = fp32_fma_rate(mode=mode)
    print(f"mode {mode}: {rate:.1f} TFLOP/s ({rate / nominal:.1%} of nominal)")
    assert 0.2 * nominal < rate < 1.02 * nominal, (rate, nominal)

"""The integer min/max throughput probe (nbldpc_probe_minmax): every form
launches, fills the device and reports the min-max pairs it performs."""
import pytest
import torch

from paper_2508_03567_gb300 import binding

pytestmark = pytest.mark.gpu

FORMS = (binding.NBLDPC_PROBE_ALU, binding.NBLDPC_PROBE_FMA_1_8, binding.NBLDPC_PROBE_FMA_3_8,
         binding.NBLDPC_PROBE_FMA_4_8, binding.NBLDPC_PROBE_FMA_3_8_SHFL, binding.NBLDPC_PROBE_CONV_64,
         binding.NBLDPC_PROBE_CONV_256)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("form", FORMS)
def test_probe_form_runs_and_counts_pairs(form):
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    pairs, blocks = binding.nbldpc_probe_minmax(form, 3, sink)
    torch.cuda.synchronize()
    assert blocks >= sms and blocks % sms == 0
    if form in (binding.NBLDPC_PROBE_CONV_64, binding.NBLDPC_PROBE_CONV_256):
        q = 64 if form == binding.NBLDPC_PROBE_CONV_64 else 256
        per_thread = q * q / (16 if q == 64 else 32)      # q^2 pairs per convolution of a lane group
    else:
        per_thread = 4 * 32 * 2                            # 4 steps x 32 packed maxima x 2 symbols
    assert pairs == per_thread * 3 * blocks * 256
    assert int(sink.item()) == 0                           # the sink is never hit for values <= 255


def test_probe_rejects_bad_arguments():
    sink = torch.zeros(1, dtype=torch.int32, device="cuda")
    for form, rounds in ((99, 1), (binding.NBLDPC_PROBE_ALU, 0)):
        with pytest.raises(binding.NbldpcError) as ei:
            binding.nbldpc_probe_minmax(form, rounds, sink)
        assert ei.value.status == binding.NBLDPC_ERR_ARG

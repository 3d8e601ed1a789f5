"""The library's automatic choices, seen through what a call reports: with
grain 0 the number of work units shows the grain the library picked, which
must follow the rule the header states (about two units per resident sweep
warp, the nearest power of two in [512, 8192]; 64 warps per SM when the
state array takes at most half the L2, else 48)."""
import ctypes

import pytest
import torch

import graphgen as gg
from tests.conftest import cuda_ok

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def skp():
    import paper_2507_04420_gb300 as m
    torch.cuda.set_device(0)
    return m


def _rule(items, sms, lean):
    target = items // (2 * sms * (64 if lean else 48))
    grain = 512
    while grain < 8192 and grain * 1414 < target * 1000:
        grain *= 2
    return grain


@pytest.mark.parametrize("bits", [2, 8, 32])
def test_grain_zero_follows_the_stated_rule(skp, bits):
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    l2 = ctypes.c_int(0)    # cudaDevAttrL2CacheSize, the attribute the library reads
    assert ctypes.CDLL("libcudart.so").cudaDeviceGetAttribute(ctypes.byref(l2), 38, 0) == 0
    l2 = l2.value
    for g in (gg.path(3000), gg.erdos_renyi(100_000, 1_000_000, seed=1), gg.rmat(18, 16, seed=2),
              gg.rmat(20, 16, seed=3), gg.grid(2048, 2048)):
        state_bytes = 4 * g.n if bits == 32 else 4 * -(-g.n // (32 // bits))
        lean = 2 * state_bytes <= l2
        items = g.n + g.nnz
        grain = _rule(items, sms, lean)
        mate = torch.empty(g.n, dtype=torch.int32, device="cuda")
        with skp.Graph(g.offsets.cuda(), g.nbrs.cuda()) as h:
            h.skipper(mate=mate, status_bits=bits, grain=0, timing=1)
            assert h.timing()["units"] == -(-items // grain), (g.n, bits, grain)
            assert h.validate(mate).flags == 0

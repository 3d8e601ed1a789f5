"""Host-side admission logic of the server (no GPU needed)."""
from paper_2507_04420_gb300.server import device_bytes, plan_admission


def test_admission_in_arrival_order_without_overtaking():
    sizes = [100, 300, 50, 50]
    assert plan_admission(sizes, used=0, budget=1000, max_graphs=10) == (4, 500)
    # the second request does not fit: nothing behind it is admitted either
    assert plan_admission(sizes, used=700, budget=1000, max_graphs=10) == (1, 100)
    assert plan_admission(sizes, used=950, budget=1000, max_graphs=10) == (0, 0)
    assert plan_admission(sizes, used=0, budget=1000, max_graphs=2) == (2, 400)
    assert plan_admission([], used=0, budget=10, max_graphs=10) == (0, 0)


def test_device_bytes_counts_csr_and_mate():
    b = device_bytes(1000, 8000)
    assert b >= 8 * 1001 + 4 * 8000 + 4 * 1000
    assert b % 512 == 0
    assert device_bytes(0, 0) > 0


def test_device_bytes_in_place_leaves_the_csr_on_the_host():
    for n, nnz in ((1000, 8000), (1 << 20, 1 << 24), (1, 0)):
        copied, in_place = device_bytes(n, nnz), device_bytes(n, nnz, in_place=True)
        r = lambda b: (b + 511) // 512 * 512
        assert copied - in_place == r(8 * (n + 1)) + r(4 * max(nnz, 1))
        assert in_place >= 4 * n and in_place % 512 == 0


def test_native_server_needs_a_device():
    """Creating the native server without a GPU fails with MM_ERR_CUDA (no CPU fallback)."""
    import ctypes
    import torch
    from paper_2507_04420_gb300 import lib
    from paper_2507_04420_gb300._native import ServerConfig
    if torch.cuda.is_available():
        return
    cfg = ServerConfig()
    assert lib.mm_server_default_config(ctypes.byref(cfg)) == 0
    assert (cfg.slots, cfg.validate, cfg.in_place_max_nnz, cfg.max_graphs_per_tick) == (2, 1, 1 << 20, 4096)
    h = ctypes.c_void_p()
    assert lib.mm_server_create(ctypes.byref(cfg), ctypes.byref(h)) == 3
    assert lib.mm_server_create(None, ctypes.byref(h)) == 1
    cfg.slots = 3
    assert lib.mm_server_create(ctypes.byref(cfg), ctypes.byref(h)) == 1

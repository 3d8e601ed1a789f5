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

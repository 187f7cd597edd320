"""Host logic of the serving loop: first-come-first-served admission against a
device-memory budget (no GPU)."""
import pytest

from paper_2607_00199_b300 import inputs
from paper_2607_00199_b300.serve import Admission, predicted_device_bytes


def test_fifo_and_budget():
    a = Admission(1000)
    for i in range(5):
        a.arrive({'id': i}, 400)
    got = [r['id'] for r, _ in a.admit()]
    assert got == [0, 1] and a.used == 800
    assert a.admit() == []                       # the head does not fit: nothing overtakes it
    a.release(400)
    assert [r['id'] for r, _ in a.admit()] == [2]
    assert a.peak <= a.budget


def test_head_of_line_is_kept():
    a = Admission(1000)
    a.arrive({'id': 0}, 900)
    a.arrive({'id': 1}, 500)
    a.arrive({'id': 2}, 50)
    assert [r['id'] for r, _ in a.admit()] == [0]
    # request 2 would fit but must wait behind request 1 (arrival order)
    assert a.admit() == []
    a.release(900)
    assert [r['id'] for r, _ in a.admit()] == [1, 2]


def test_max_active_and_oversize():
    a = Admission(10 ** 9, max_active=2)
    for i in range(4):
        a.arrive({'id': i}, 10)
    assert len(a.admit()) == 2
    with pytest.raises(ValueError):
        a.arrive({'id': 9}, 10 ** 10)


def test_request_stream_and_memory_model():
    reqs = inputs.serving_requests(256, rate=50.0, seed=1)
    assert len(reqs) == 256
    arr = [r['arrival'] for r in reqs]
    assert arr == sorted(arr) and 2.0 < arr[-1] < 10.0          # mean rate 50/s
    assert {r['K'] for r in reqs} <= {2048, 8192, 32768, 131072}
    assert {r['N'] for r in reqs} <= {2, 3, 4, 5}
    for r in reqs:
        assert 2 * r['n'] ** 2 == r['K']
        assert 0.01 <= r['A'] <= 0.08 and 0.5 <= r['T'] <= 2.0 and 100 <= r['Re'] <= 2000
    # the predicted footprint grows with K and N
    assert predicted_device_bytes(131072, 5) > predicted_device_bytes(131072, 4) > predicted_device_bytes(2048, 4)

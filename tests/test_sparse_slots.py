"""Slot arithmetic of sparse checkpoint buffers (host-only C ABI functions)."""
import pytest

from paper_2301_01396_gb300 import binding


@pytest.mark.parametrize("steps,stride", [(0, 1), (1, 1), (10, 1), (10, 3), (10, 5), (10, 10), (10, 20), (60, 8),
                                          (61, 8), (900, 30)])
def test_slots_are_the_multiples_of_stride_and_the_last_step(steps, stride):
    stored = [n for n in range(steps + 1) if n % stride == 0 or n == steps]
    assert binding.sparse_slots(steps, stride) == len(stored)
    slots = [binding.sparse_slot(steps, stride, n) for n in range(steps + 1)]
    assert [n for n, s in enumerate(slots) if s >= 0] == stored
    assert [s for s in slots if s >= 0] == list(range(len(stored)))


def test_invalid_arguments():
    assert binding.sparse_slots(-1, 1) == -1
    assert binding.sparse_slots(10, 0) == -1
    assert binding.sparse_slot(10, 3, 11) == -1
    assert binding.sparse_slot(10, 3, -1) == -1

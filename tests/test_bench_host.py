"""Host-side helpers of bench.py (no GPU): the sysfs CPU-list parser and the
GPU-local placement block, which must be a no-op where there is no device."""
import os

import bench


def test_cpulist_parses_ranges_and_singles():
    assert bench._cpulist("0-3,8,10-11\n") == {0, 1, 2, 3, 8, 10, 11}
    assert bench._cpulist("5") == {5}
    assert bench._cpulist("") == set()


def test_near_gpu_memory_is_a_no_op_without_a_device():
    before = os.sched_getaffinity(0)
    with bench.near_gpu_memory(0) as placement:
        inside = os.sched_getaffinity(0)
    assert os.sched_getaffinity(0) == before
    if placement.cpus is None:          # no device properties or no sysfs entry here
        assert inside == before

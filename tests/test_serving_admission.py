"""Admission control of the serving engine, on the host with a fake device
memory budget (no GPU)."""
from paper_1909_07226_gb300 import serving
from paper_1909_07226_gb300 import synthetic as syn


def test_admission_respects_budget_and_slots():
    a = serving.Admission(budget_bytes=100, max_slots=3)
    assert a.admit(1, 40) and a.admit(2, 40)
    assert not a.admit(3, 30)          # 110 > 100: waits for memory
    assert a.admit(4, 20)              # fits
    assert not a.admit(5, 1)           # no slot left
    a.release(2)
    assert a.admit(3, 30) and a.used_bytes == 90
    assert not a.admit(3, 1)           # already admitted
    a.release(1)
    a.release(3)
    a.release(4)
    assert a.used_bytes == 0 and not a.active


def test_job_bytes_and_trace():
    wls = syn.make_batched_jobs(6, seed=5, scale_t=0.05)
    for w in wls:
        need = serving.job_bytes(w)
        assert need >= 2 * w.n_vis * 32 + 3 * w.grid_size ** 2 * 32
    tr = serving.make_trace(wls, 50.0, ("cycle", "grid", "degrid"), seed=3)
    arr = [j.arrival for j in tr]
    assert arr == sorted(arr) and arr[0] > 0
    assert {j.kind for j in tr} <= {"cycle", "grid", "degrid"}
    assert all(j.n_steps == (5 if j.kind == "cycle" else 1) for j in tr)
    # identical traces from the same seed
    tr2 = serving.make_trace(wls, 50.0, ("cycle", "grid", "degrid"), seed=3)
    assert [(j.kind, j.arrival, j.seed) for j in tr] == [(j.kind, j.arrival, j.seed) for j in tr2]

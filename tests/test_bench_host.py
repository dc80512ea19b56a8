"""Host logic of the benchmark and the binding, CPU only: the DRAM-traffic figure is taken
only from a capture of the same kernel source and launch shape, and a solve's per-seed
stats read lazily from the C array behave as a sequence of dicts."""
import ctypes
import hashlib
import importlib.util
import json
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


TUNING = {"t1": 32, "t2": 128, "chunk": 512, "schedule": 4, "hub_degree": 128}


def _files(tmp_path, src=b"kernel source", captures=None, kernel="k_batch_rounds", sha=None):
    ks = tmp_path / "batched.cu"
    ks.write_bytes(src)
    tj = {"kernel": kernel, "source_sha256": sha or hashlib.sha256(src).hexdigest(), "graph": "rmat20",
          "seeds": 128, "captures": captures if captures is not None else [
              {"tuning": dict(TUNING, hub_degree=64), "bytes_per_edge": 29.0},
              {"tuning": dict(TUNING), "bytes_per_edge": 30.0}]}
    tp = tmp_path / "traffic.json"
    tp.write_text(json.dumps(tj))
    return str(tp), str(ks)


def test_traffic_takes_the_capture_of_the_launch_tuning(tmp_path):
    b = _bench()
    tp, ks = _files(tmp_path)
    # blocks_per_sm is not part of the match (the grid follows the occupancy)
    t, note = b.traffic_from_capture(tp, ks, dict(TUNING, blocks_per_sm=0), 1e9)
    assert t == pytest.approx(30.0e9) and "30.00 B per pushed edge" in note
    t, _ = b.traffic_from_capture(tp, ks, dict(TUNING, hub_degree=64, blocks_per_sm=3), 2e9)
    assert t == pytest.approx(58.0e9)


@pytest.mark.parametrize("case", ["other_tuning", "source_changed", "other_kernel", "missing"])
def test_traffic_is_null_without_a_matching_capture(tmp_path, case):
    b = _bench()
    tp, ks = _files(tmp_path, kernel="k_other" if case == "other_kernel" else "k_batch_rounds",
                    sha=("0" * 64) if case == "source_changed" else None)
    tuning = dict(TUNING, hub_degree=160) if case == "other_tuning" else dict(TUNING)
    if case == "missing":
        tp = str(tmp_path / "absent.json")
    assert b.traffic_from_capture(tp, ks, tuning, 1e9) == (None, None)


def test_committed_captures_are_consistent():
    """profiles/traffic.json: each capture's bytes per edge is its DRAM bytes over the small
    case's pushed edges, and its command keeps the clocks alone."""
    tj = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert tj["kernel"] == "k_batch_rounds" and len(tj["source_sha256"]) == 64
    for c in tj["captures"]:
        assert c["bytes_per_edge"] == pytest.approx((c["dram_bytes_read"] + c["dram_bytes_write"])
                                                    / tj["edges_per_launch"])
        assert "--clock-control none" in c["command"]


def test_stats_list_is_a_lazy_sequence_of_dicts():
    import paper_2410_21634_gb300 as gde
    arr = (gde.Stats * 4)()
    for i in range(4):
        arr[i].rounds = 10 + i
        arr[i].fallback = i % 2
    st = gde.StatsList(arr, 3)  # a batch of 3 in a larger buffer
    assert len(st) == 3
    assert st[0]["rounds"] == 10 and st[-1]["rounds"] == 12 and st[1]["fallback"] == 1
    assert [s["rounds"] for s in st] == [10, 11, 12]
    assert [s["rounds"] for s in st[1:]] == [11, 12]
    assert sum(1 for s in st if s["fallback"]) == 1
    assert isinstance(st[0], dict) and isinstance(st[0]["rounds"], int)
    with pytest.raises(IndexError):
        st[3]
    with pytest.raises(IndexError):
        st[-4]
    assert json.loads(json.dumps(list(st)))[2]["rounds"] == 12
    assert ctypes.sizeof(gde.Stats) == 48

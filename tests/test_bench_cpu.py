"""Host-side logic of bench.py (no GPU): the max-over-ranks timing reduction
with two gloo ranks, the reference arm (the CPU oracle on a bounded sample),
and its single-printer rule under torchrun-style environments."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank, bench.max_over_ranks(1.5 + rank)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import socket
    import torch.multiprocessing as mp
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert got == [(0, 2.5), (1, 2.5)]


def test_max_over_ranks_without_group_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25) == 3.25


def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "2", "--warmup", "3", "--ref-scale", "9"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert isinstance(d["cpu_baseline"]["cpu_model"], str) and d["cpu_baseline"]["cpu_model"]
    assert d["cpu_baseline"]["host_cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_only_rank0_prints():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--ref-scale", "8"], capture_output=True, text=True,
                       timeout=300, cwd=ROOT, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_algorithmic_bytes_formula():
    sys.path.insert(0, ROOT)
    import bench
    # 4 bytes per merge element, 8 per live edge, 16 per triangle, 8 per row pointer
    assert bench.algorithmic_bytes(n=3, live=2, merge=10, tris=1) == 40 + 16 + 16 + 32


def test_traffic_record_is_bound_to_the_profiled_source_and_workload(tmp_path, monkeypatch):
    """An ncu traffic record is used only for the kernel source it was captured
    on (its sha256) and for its own workload and K; a record of a changed
    source is returned as stale."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "paper_2009_07929_gb300" / "csrc" / "support_balanced.cu"
    src.parent.mkdir(parents=True)
    src.write_bytes(b"// kernel source as captured\n")
    shape = src.parent / "support_shape.cuh"
    shape.write_bytes(b"// per-shape part\n")
    (tmp_path / "profiles").mkdir()
    rec = {"kernel": "support_kernel", "workload": "rmat20 K=3 round 1",
           "source_sha256": bench.kernel_source_sha256(str(tmp_path)),
           "dram_bytes_per_launch": 123456}
    (tmp_path / "profiles" / "support_traffic.json").write_text(json.dumps([rec]))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    r, fresh = bench.traffic_record("rmat20", 3)
    assert fresh and r["dram_bytes_per_launch"] == 123456
    assert bench.traffic_record("rmat20", 4) == (None, False)
    assert bench.traffic_record("rmat23c", 3) == (None, False)
    shape.write_bytes(b"// per-shape part changed after the capture\n")
    r, fresh = bench.traffic_record("rmat20", 3)
    assert r is not None and not fresh


def _work_by_loops(rp, col, light):
    """support_work's quantities by plain loops over the edges."""
    n = len(rp) - 1
    W = probes = segs = 0
    staged = set()
    for i in range(n):
        for e in range(rp[i], rp[i + 1]):
            k = col[e]
            t = rp[i + 1] - e - 1
            d = rp[k + 1] - rp[k]
            W += t + d
            if t + d > light and min(t, d) > 0:
                probes += min(t, d)
                segs += 1
                staged.add(k if t < d else i)
    return {"W": W, "probes": probes, "segments": segs, "active_rows": len(staged),
            "staged": sum(rp[r + 1] - rp[r] for r in staged)}


@pytest.mark.parametrize("light", [0, 4, 64])
def test_support_work_counts_match_loops(light):
    sys.path.insert(0, ROOT)
    import bench
    import graphgen as gg
    for g in (gg.rmat(9, 16, seed=3), gg.er(300, 3000, seed=1), gg.complete(40), gg.star(30),
              gg.empty(5)):
        want = _work_by_loops(g.row_ptr.tolist(), g.col.tolist(), light)
        assert bench.support_work(g.row_ptr, g.col, light) == want


def test_design_bytes_formula():
    sys.path.insert(0, ROOT)
    import bench
    w = {"probes": 10, "staged": 5, "segments": 2, "active_rows": 1, "W": 99}
    assert bench.design_bytes(w, 3) == 40 + 60 + 24 + 56 + 16


def test_clock_summary_uses_samples_inside_the_timed_region():
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    row = "0, {sm}, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, {cap}"
    c.lines = [(1.0, row.format(sm=1200, cap="Not Active"))]  # before the region
    c.t_start = 2.0
    assert c.summary()["sm_mhz"] == 1200 and c.summary()["samples"] == 1  # only one: kept
    c.lines += [(2.1, row.format(sm=2070, cap="Active")), (2.3, row.format(sm=2050, cap="Not Active"))]
    s = c.summary()
    assert s["sm_mhz"] == 2060 and s["sm_max_mhz"] == 2070 and s["samples"] == 2
    assert s["reasons"] == ["sw_power_cap"]
    # a sample taken after the region ended is not part of it
    c.t_end = 2.5
    c.lines.append((2.7, row.format(sm=900, cap="Not Active")))
    assert c.summary()["sm_mhz"] == 2060 and c.summary()["samples"] == 2
    c.lines = []
    assert c.summary()["reasons"] == ["unsampled"]

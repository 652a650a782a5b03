"""Host-side pieces of bench.py: the max/sum reduction over ranks (two gloo
ranks on CPU), the reference arm on a non-zero rank, clock-sample parsing,
and the profile-summary staleness check."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mx, sm = bench.reduce_over_ranks([1.0 + rank, 10.0 * rank], [2.0 + rank], "cpu")
    q.put((rank, mx, sm))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_over_ranks_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, sm in out:
        assert mx == [2.0, 10.0] and sm == [5.0]


def test_single_rank_reduce_is_identity():
    import bench
    assert bench.reduce_over_ranks([3.0], [4.0], "cpu") == ([3.0], [4.0])


def test_reference_arm_nonzero_rank_is_silent():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_parse_clock_lines():
    import bench
    lines = ["1965, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
             "2070, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
             "2010, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
             "garbage"]
    c = bench.parse_clock_lines(lines)
    assert c == {"sm_mhz": 2010.0, "sm_max_mhz": 2070.0, "samples": 3, "reasons": ["sw_power_cap"]}
    assert bench.parse_clock_lines([]) is None


def test_profiled_traffic_tracks_kernel_sources(tmp_path, monkeypatch):
    import bench
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "hop_dw_24x24x24x48.md").write_text(
        f"- kernel_sources_sha256_16: `{bench.kernel_hash()}`\n- dram_bytes_per_launch: 123\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "paper_2409_03030_gb300").symlink_to(os.path.join(ROOT, "paper_2409_03030_gb300"))
    assert bench.profiled_traffic() == 123.0
    (prof / "hop_dw_24x24x24x48.md").write_text(
        "- kernel_sources_sha256_16: `0000000000000000`\n- dram_bytes_per_launch: 123\n")
    assert bench.profiled_traffic() is None


def test_kernel_hash_covers_the_double_word_hop_sources():
    """The hash that ties the committed ncu traffic to the double-word hop
    covers exactly the kernel's translation unit and every project header it
    reaches, less the two headers that serve only the low-precision kernels:
    a header added to that chain must join the list, or a changed kernel would
    keep reporting stale traffic."""
    import re
    import bench
    csrc = os.path.join(ROOT, "paper_2409_03030_gb300", "csrc")

    def includes(name):
        with open(os.path.join(csrc, name)) as fh:
            return [m for m in re.findall(r'#include\s+"([^"]+)"', fh.read())
                    if os.path.exists(os.path.join(csrc, m))]

    reached, todo = set(), ["dslash.cu"]
    while todo:
        f = todo.pop()
        if f in reached or f in ("hop_lp.cuh", "cg_steps.cuh"):
            continue
        reached.add(f)
        todo.extend(includes(f))
    assert reached == set(bench.HOP_KERNEL_SOURCES), sorted(reached ^ set(bench.HOP_KERNEL_SOURCES))

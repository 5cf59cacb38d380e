"""bench.py host logic on the CPU: the multi-rank reduction (gloo, 2 ranks), the whole-job
rate, and the reference arm's JSON line (the CPU oracle on the 4^4 workload)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.reduce_max(1.0 + rank, world, "cpu")  # rank r was r + 1 seconds slow
    dist.barrier()
    with open(out + f".{rank}", "w") as fh:
        fh.write(repr(t))
    dist.destroy_process_group()


def test_two_rank_max_and_weak_scaling(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    out = str(tmp_path / "r")
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    vals = [float(open(out + f".{r}").read()) for r in range(2)]
    assert vals == [2.0, 2.0]  # both ranks see the slowest rank's time
    # 10 solves per rank on 2 ranks in 2 s (the slowest rank) is 10 solves/s for the job
    assert bench.whole_job_rate(10, 2, 2.0) == 10.0
    assert bench.reduce_max(3.5, 1, "cpu") == 3.5


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "4^4", "--steps", "2", "--warmup", "3", "--ref-seconds", "0.2",
                        "--ref-iters", "40"], capture_output=True, text=True, timeout=300,
                       cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "solves/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["higher_is_better"] is True
    assert line["metric"] == bench.METRIC and line["warmup"] == 3 and line["steps"] == 2
    assert 0 < line["sample_ms_per_step"] < 60e3  # the bounded sample, not the modelled solve


def test_trimmed_mean_drops_stray_launches():
    import bench
    ts = [14.3e-6] * 18 + [148e-6, 14.1e-6]
    assert abs(bench.trimmed_mean(ts) - 14.3e-6) < 1e-12
    assert bench.trimmed_mean([2.0, 4.0]) == 3.0


def test_hopping_byte_counts():
    """Algorithmic and naive bytes per output site of one half-lattice hopping application:
    one input spinor, the 8 links and one output (algorithmic), eight neighbour spinors instead of
    one (naive), for every storage form with 18/12/8-real links."""
    import bench
    F64, F32, F16 = 0, 1, 2
    expect = {(F64, 18): (1536, 2880), (F64, 12): (1152, 2496), (F32, 18): (768, 1440),
              (F32, 12): (576, 1248), (F16, 12): (296, 660), (F16, 8): (232, 596)}
    for (prec, nreal), (alg, naive) in expect.items():
        assert bench.hop_bytes_per_site(prec, nreal) == alg
        assert bench.hop_naive_bytes_per_site(prec, nreal) == naive


def test_traffic_lines_of_the_committed_profiles():
    """Each `bench-traffic:` line under profiles/ names a known form and lattice, a kernel choice
    and a 12-digit source digest, and its DRAM bytes lie within 10% of the algorithmic bytes of one
    launch of that form on that lattice (so a figure the bench reports as roofline.traffic is one
    launch's worth); the headline form's line is found by ncu_traffic when its digest is current."""
    import glob
    import re
    import bench
    from paper_0905_3331_gb300 import inputs
    pat = re.compile(r"bench-traffic: form=(\S+) lattice=(\S+) kernel=(\d+) sources=([0-9a-f]+) bytes=(\d+)")
    found = 0
    for path in glob.glob(os.path.join(ROOT, "profiles", "*.md")):
        for line in open(path):
            m = pat.search(line)
            if not m:
                continue
            found += 1
            form, lattice, kernel, digest, nbytes = m.groups()
            prec, nreal = bench.parse_sloppy(form)
            w = inputs.WORKLOADS[lattice]
            alg = bench.hop_bytes_per_site(prec, nreal) * (w.V // 2)
            assert len(digest) == 12 and int(kernel) in (1, 2, 3, 4, 5)
            assert abs(int(nbytes) - alg) < 0.1 * alg, (path, form, lattice, nbytes, alg)
            if digest == bench.kernel_sources_hash(prec):
                assert bench.ncu_traffic(form, lattice, int(kernel), prec)[0] == float(nbytes)
    assert found >= 1

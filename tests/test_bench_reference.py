"""bench.py's reference arm (the oracle on the host cores) reports the same
workload and config as the main line, so the two lines compare like with
like; its value comes from the same bounded sample the main line's
cpu_baseline times."""
import json
import os
import subprocess
import sys

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_config_matches_main_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "jacobi2d", "--steps", "2", "--warmup", "3"],
                       capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    wl = bench.make_workload("jacobi2d")
    wl.host_setup()
    assert line["config"] == json.loads(json.dumps(bench._config(wl, 1)))
    assert line["metric"] == wl.metric and line["unit"] == wl.unit
    assert line["cpu_baseline"]["value"] == line["value"] > 0


def test_default_workload_is_the_largest_f64_configuration():
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert 'ap.add_argument("--workload", default="heat3d")' in src
    wl = bench.make_workload("heat3d")
    assert wl.shape == (512, 512, 512) and wl.T == 50 and wl.dtype == "f64"
    assert wl.bc == "periodic"


def test_every_workload_states_its_cpu_sample():
    # batch2d's sample size depends on its drawn instance sides (host_setup)
    for name in ("heat3d", "jacobi2d", "map_reduce_f32", "map_reduce_f64",
                 "map_reduce_rows_f32", "tanh_adjoint", "tanh_adjoint_2d"):
        wl = bench.make_workload(name)
        assert wl.cpu_desc and wl.cpu_scale >= 1.0


def test_tiled_reverse_workload_traffic_model_matches_its_plan():
    """tanh_adjoint_2d's algorithmic bytes assume one forward launch per
    stored checkpoint (each reads and writes a state) and one reverse launch
    per chunk (each reads two states and writes one); the library's plan of
    that exact program (dcp_prepare_adjoint, no GPU) has those launches."""
    wl = bench.make_workload("tanh_adjoint_2d", 256)
    g = wl._graph(wl.DEPTH, True)
    launches = g.prepare_adjoint()["adjoint"]["launches"]
    chunks = (wl.T + wl.DEPTH - 1) // wl.DEPTH
    fwd = [l for l in launches if l["phase"] == "forward"]
    rev = [l for l in launches if l["phase"] == "reverse" and l["kernel"].startswith("dcp_adj_")]
    assert len(fwd) == chunks - 1 and len(rev) == chunks
    wl.n_launch = len(launches)
    states = 2 * (chunks - 1) + 3 * chunks + 1
    assert abs(wl.roof()["bytes"] * wl.n_launch - states * 256 * 256 * 4) < 1.0

"""Host logic of the tile planner (plan_tiles in csrc/pfc_host.h), compiled as a small host
program: every plan for the supported shapes keeps the invariants the kernels rely on."""
import itertools
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SMEM_MAX = 232448


@pytest.fixture(scope="module")
def planner(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path_factory.mktemp("planner") / "plan_dump")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-o", exe, os.path.join(ROOT, "tests", "host", "plan_dump.cu")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]

    def run(cases, all_candidates=False, sched=None):
        args = [str(v) for c in cases for v in c]
        env = dict(os.environ)
        env.pop("PFC_TILE", None)
        env.pop("PFC_ROW_CLUSTER", None)
        if all_candidates:
            env["PLAN_DUMP_ALL"] = "1"
        if sched is not None:
            env["PLAN_DUMP_SCHED"] = str(sched)
        out = subprocess.run([exe, *args], capture_output=True, text=True, check=True, env=env).stdout
        return [json.loads(l) for l in out.splitlines()]
    return run


def _cases():
    dims = [16, 32, 64, 128, 256, 512, 1024, 2048, 4096]
    cases = []
    for nx, ny in itertools.product(dims, dims):
        for vb in (8, 16):
            cases.append((nx, ny, 1, vb, 2, 1))
    for n in (16, 32, 64, 128, 256, 512):
        for vb in (8, 16):
            for ntile in (2, 3):
                cases.append((n, n, n, vb, ntile, 1))
    cases += [(512, 256, 256, 8, 2, 1), (4096, 16, 16, 8, 2, 1), (16, 16, 4096, 8, 2, 1), (64, 64, 1, 8, 2, 400)]
    # grids beyond the two-pass tilings (three-pass schedule)
    cases += [(1024, 1024, 1024, 8, 2, 1), (1024, 1024, 1024, 16, 2, 1), (2048, 2048, 2048, 8, 2, 1),
              (2048, 2048, 2048, 16, 2, 1), (4096, 4096, 4096, 8, 2, 1), (4096, 1024, 1024, 8, 2, 1),
              (1024, 2048, 2048, 8, 2, 1)]
    return cases


def _check_plan(p):
    nx, ny, nz, vb = p["nx"], p["ny"], p["nz"], p["vb"]
    M = nx // 2
    assert p["M"] == M
    assert p["P"] == p["Py"] * p["Pz"] and p["Q"] == p["Qy"] * p["Qz"]
    assert p["R"] == p["Ry"] * p["Rz"] and p["QR"] == p["R"] * p["Q"]
    assert p["Py"] * p["Ry"] * p["Qy"] == ny and p["Pz"] * p["Rz"] * p["Qz"] == nz
    assert p["Py"] in (1, 2, 4, 8) and p["Pz"] in (1, 2, 4, 8)
    assert p["Ry"] in (1, 2, 4, 8) and p["Rz"] in (1, 2, 4, 8)
    assert p["Qy"] == 1 or p["Qy"] >= 8
    assert p["Qz"] == 1 or p["Qz"] >= 8
    assert nz > 1 or (p["Pz"] == 1 and p["Rz"] == 1)
    if p["R"] > 1:   # three-pass line tiles have both axes of at least 8 (one in 2D)
        assert p["Qy"] >= 8 and (nz == 1 or p["Qz"] >= 8)
    # X' rows: every bin, a whole number of tiles, 16-byte aligned rows
    assert p["xs"] >= M + 1 and p["xs"] % p["W"] == 0 and p["ncg"] * p["W"] == p["xs"]
    assert (p["xs"] * vb) % 16 == 0
    assert p["nhalf"] == p["P"] * p["QR"] * p["xs"]
    # line tiles: one padding row per 8 tile rows, 8 elements per thread
    assert p["tsz"] == (p["Q"] + p["Q"] // 8) * p["W"]
    assert p["nt_line"] * 8 == p["Q"] * p["W"]
    assert p["nt_line"] <= (1024 if vb == 8 else 512)
    assert p["smem_line"] == p["ntile"] * p["tsz"] * vb <= SMEM_MAX
    # row blocks: rows of M + 1 bins (stride a multiple of 16 for the XOR swizzle)
    assert p["rs"] >= M + 1 and p["rs"] % 16 == 0
    assert p["nt_row"] <= 512 and p["nt_row"] % max(1, M // 8) == 0
    assert p["smem_row"] <= SMEM_MAX
    assert p["QR"] % p["gpc"] == 0
    # clustered psi^3 rows: FP32 only, at the row lengths the kernels are compiled for
    if p["row_cs"]:
        assert vb == 8 and p["row_cs"] == 2 and p["gpc"] == 1
        assert (p["Pz"] == 1 and p["Py"] == 8 and M == 2048) or (p["Pz"] == 8 and M in (256, 512, 1024))
        assert p["smem_row_cs"] <= SMEM_MAX // 2   # two blocks per SM
        assert p["nt_row_cs"] <= 512


def test_plans_keep_the_kernel_invariants(planner):
    plans = planner(_cases())
    assert len(plans) == len(_cases())
    for p in plans:
        # every grid has a plan: two-pass where a row group and two line tiles fit, else
        # three-pass; only grids whose arrays exceed the GPU's 288 GB anyway have none (the
        # middle pass takes at most 8 x 8 points)
        if (p["nx"], p["ny"], p["nz"], p["vb"]) in ((2048, 2048, 2048, 16), (4096, 4096, 4096, 8)):
            assert not p["ok"]
            continue
        assert p["ok"], p
        _check_plan(p)
        if p["R"] > 1:
            assert (p["vb"] == 16 and p["nz"] >= 512) or p["nz"] >= 1024 or p["nx"] * p["ny"] * p["nz"] >= 2 ** 30


def test_every_autotune_candidate_keeps_the_kernel_invariants(planner):
    """The autotuner times tilings other than the planner's: each must satisfy the same
    invariants, and the first candidate must be the planner's own choice."""
    cases = [c for c in _cases() if c[0] * c[1] * c[2] <= 512 ** 3]
    chosen = {tuple(c): p for c, p in zip(cases, planner(cases))}
    allc = planner(cases, all_candidates=True)
    assert allc
    seen_first = set()
    for p in allc:
        assert p["ok"], p
        _check_plan(p)
        key = (p["nx"], p["ny"], p["nz"], p["vb"], p["ntile"], p["inst"])
        if p["cand"] == 0 and key not in seen_first:
            seen_first.add(key)
            ref = chosen[key]
            for k in ("Py", "Pz", "W", "row_cs"):
                assert p[k] == ref[k], (key, k)
    # the clustered grids also offer the single-block row pass
    c4096 = [p for p in planner([(4096, 4096, 1, 8, 2, 1)], all_candidates=True) if p["cand"] == 0]
    assert [p["row_cs"] for p in c4096] == [2, 0]


def test_bench_and_config_plans(planner):
    p, q, single, batch = planner([(4096, 4096, 1, 8, 2, 1), (512, 512, 512, 8, 2, 1),
                                   (64, 64, 1, 8, 2, 1), (64, 64, 1, 8, 2, 400)])
    assert (p["Py"], p["Qy"], p["W"], p["nt_line"], p["row_cs"]) == (8, 512, 4, 256, 2)
    assert (q["Py"], q["Pz"], q["W"], q["row_cs"]) == (8, 8, 2, 2)
    # a small grid alone keeps one row block per SM; as a batch class it packs row groups
    assert single["gpc"] == 1 and batch["gpc"] > 1


def test_autotune_cache_file_round_trip(tmp_path):
    """The autotune cache (host code): entries are valid JSON lines, a lookup finds the last entry
    for its key, other keys and malformed lines are skipped."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "tune_cache")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-o", exe, os.path.join(ROOT, "tests", "host", "tune_cache.cu")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    path = tmp_path / "tiles.jsonl"
    path.write_text("not json\n{\"key\": \"other\"}\n")
    out = subprocess.run([exe, str(path)], capture_output=True, text=True, check=True).stdout
    a, b, c = [json.loads(l) for l in out.splitlines()]
    assert a["found"] and (a["Py"], a["Pz"], a["W"], a["cluster"]) == (8, 1, 2, 1) and a["ms"] == 0.16
    assert b["found"] and (b["Py"], b["Pz"], b["W"], b["cluster"]) == (2, 2, 8, 0)
    assert not c["found"]
    entries = [json.loads(l) for l in path.read_text().splitlines()[2:]]
    assert [e["key"] for e in entries] == ["1x4096x4096 prec1 fields1 NVIDIA_GB300",
                                           "256x256x256 prec1 fields2 NVIDIA_GB300",
                                           "1x4096x4096 prec1 fields1 NVIDIA_GB300"]
    assert entries[1] == {"key": "256x256x256 prec1 fields2 NVIDIA_GB300", "Py": 2, "Pz": 2, "W": 8,
                          "cluster": 0, "Ry": 1, "Rz": 1, "ms_per_step": 0.556376}


def test_three_pass_plans(planner):
    """Grids with no two-pass tiling get three-pass plans; a two-pass grid keeps its plan and also
    lists three-pass candidates for the autotuner."""
    f64_512, f32_1024, f32_2048 = planner([(512, 512, 512, 16, 2, 1), (1024, 1024, 1024, 8, 2, 1),
                                           (2048, 2048, 2048, 8, 2, 1)])
    for p in (f64_512, f32_1024, f32_2048):
        assert p["ok"] and p["R"] > 1
        _check_plan(p)
    assert f32_2048["nt_line"] <= 1024
    # 512^3 FP32 has a two-pass plan; its three-pass candidates all keep the invariants
    three = planner([(512, 512, 512, 8, 2, 1), (256, 256, 256, 16, 2, 1), (64, 128, 1, 8, 2, 1)],
                    all_candidates=True, sched=3)
    assert three and all(p["ok"] and p["R"] > 1 for p in three)
    for p in three:
        _check_plan(p)

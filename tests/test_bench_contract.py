"""bench.py's command-line contract on CPU: the oracle arm prints one JSON line with
the required keys, and the library arm fails loudly without a GPU (no CPU fallback)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, timeout=300):
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_line():
    p = _run("--impl", "reference", "--steps", "1", "--warmup", "0")
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert d["unit"] == "TFLOP/s" and d["higher_is_better"] is True and d["data"] == "synthetic"
    assert d["vs_baseline"] is None
    assert d["config"]["workload"].startswith("k40_m2000: K=40 N=40")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_library_arm_needs_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the library arm would run")
    p = _run("--steps", "1", "--warmup", "0", timeout=120)
    assert p.returncode != 0
    assert not [ln for ln in p.stdout.splitlines() if ln.startswith("{")]


def test_reference_arm_does_not_load_the_library():
    """The oracle arm times the CPU oracle alone: libgbdmrg.so stays unloaded."""
    code = ("import runpy, sys; sys.argv = ['bench.py', '--impl', 'reference', '--steps', '1', '--warmup', '0']; "
            "runpy.run_path('bench.py', run_name='__main__'); "
            "maps = open('/proc/self/maps').read(); "
            "assert 'libgbdmrg' not in maps, 'library loaded by the oracle arm'")
    p = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]


def test_oracle_sample_flops_match_the_library_count():
    """The stored algorithmic flop count of the oracle sample equals the library's host-side count."""
    import importlib.util

    import paper_1605_02611_gb300 as G
    from paper_1605_02611_gb300 import synth
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    s = bench.ORACLE_SAMPLE
    h, eri = synth.integrals(s["K"], s["seed"])
    bonds, _ = synth.random_mps(s["K"], s["N"], s["two_sz"], s["M"], s["seed"] + 1, s["spread"])
    k = s["k"]
    fl = G.sigma_flops_host(h, eri, s["N"], s["two_sz"], k, bonds[k].labels(), bonds[k + 2].labels())
    assert fl == bench.ORACLE_SAMPLE_FLOPS

"""The GPU suite's collection order and markers (checked without a GPU): every
*_gpu.py file marks its tests gpu, the files for paths first run on a GPU in a
later call (test_zy*) come after every file already run there, and
test_zz_no_alloc.py is collected last."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))


def _collected(marker):
    out = subprocess.run([sys.executable, "-m", "pytest", HERE, "--collect-only", "-q", "-m", marker],
                         capture_output=True, text=True, cwd=os.path.dirname(HERE), timeout=300)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-2000:]
    return [line.split("::")[0] for line in out.stdout.splitlines() if "::" in line]


def test_gpu_files_are_marked_and_ordered():
    gpu = _collected("gpu")
    files = list(dict.fromkeys(os.path.basename(f) for f in gpu))
    on_disk = sorted(f for f in os.listdir(HERE) if f.startswith("test_") and f.endswith(".py"))
    for f in on_disk:
        if f.endswith("_gpu.py") or f == "test_zz_no_alloc.py":
            assert f in files, f"{f} has no test marked gpu"
    assert files[-1] == "test_zz_no_alloc.py", files[-3:]
    zy = [i for i, f in enumerate(files) if f.startswith("test_zy")]
    assert zy and zy == list(range(zy[0], zy[0] + len(zy))) and zy[-1] == len(files) - 2, files
    cpu = set(os.path.basename(f) for f in _collected("not gpu"))
    assert not any(f.endswith("_gpu.py") for f in cpu), sorted(f for f in cpu if f.endswith("_gpu.py"))

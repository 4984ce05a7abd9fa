"""Both digit splits of the slicer (csrc/digits.cuh: the integer digits6 with
its BF16 encoding qbf16, and the FP32-addition split48), compiled as host C++
and checked on the CPU over random and edge-case 48-bit values: the six
digits sum exactly to the value, stay within the bounds the GEMM's exact
accumulation windows assume (|q_0| <= 256, |q_j| <= 128), and are exact BF16
values.  The same source compiles into the device kernels (slice_kernel,
slice4_kernel, slice4f_kernel)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def test_split48_properties(tmp_path):
    exe = tmp_path / "check_split48"
    subprocess.run(["g++", "-O2", "-std=c++17", "-Wall", "-Wextra", "-Werror", "-o", str(exe),
                    os.path.join(HERE, "digits", "check_split48.cpp")], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.startswith("ok ") and int(out.stdout.split()[1]) > 4_000_000

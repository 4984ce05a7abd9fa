"""The digit splits of the slicer (csrc/digits.cuh: the byte form
digit_values with pack_bf16x2, the integer digits6 / digits_n<7> with their
BF16 encoding qbf16, and the FP32-addition split48), compiled as host C++ and
checked on the CPU over random and edge-case 48-bit (and 56-bit) values: the
digits sum exactly to the value, stay within the bounds the GEMM's exact
accumulation windows assume (|q_0| <= 256, |q_j| <= 128), are exact BF16
values, and the byte form equals the integer digits bit for bit.  The same
source compiles into the device kernels (slice_kernel, slice4_kernel,
slice_group_kernel, slice4f_kernel)."""
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

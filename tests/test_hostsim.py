"""The library's host code end to end without a GPU (CPU test).

libjk.so is driven through every entry point in a child process whose CUDA
runtime is the recording stand-in of tests/hostsim/cudart_shim.c: host
memory stands in for device memory, kernels are recorded instead of run.
For each case (both engines, chunked and grouped schedules, both tile orders,
batched, host-resident, adjoint, dense densities, the density gradient,
pairings, Laplace builds, the arena-free build, the autotuner) this checks:

- the call succeeds in an arena of exactly the size the workspace query
  reports (the query and the buffers the code takes agree);
- every launch shape is within the device's limits (grid, block, dynamic
  shared memory, cluster shape);
- every tensor map obeys the TMA encoding rules (16-byte aligned base and
  strides, box at most 256 per dimension, inner box a multiple of 16 bytes
  and within the swizzle span) and addresses only memory the call owns
  (the arena or one of its inputs or outputs);
- every kernel's arguments, decoded from its signature at launch time
  (tests/hostsim/drive.py), are self-consistent with its grid, and every
  byte range its pointer arguments can touch (from the kernel's own index
  bounds) lies in memory the call owns.  Every launch must be decoded;
- with too small an arena a call fails before enqueueing any device work;
- a repeated call does no set-up and no synchronization (graph capture).
Values are not checked here: the kernels do not run.
"""
import json
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SIM = os.path.join(HERE, "hostsim")

ESIZE = {5: 8, 9: 2}            # CU_TENSOR_MAP_DATA_TYPE_INT64, _BFLOAT16
SWIZZLE_SPAN = {0: None, 1: 32, 2: 64, 3: 128}


@pytest.fixture(scope="module")
def shim_dir(tmp_path_factory):
    from paper_2608_06536_b300 import build as pkg_build
    pkg_build.build()
    d = tmp_path_factory.mktemp("cudart")
    (d / "ver.map").write_text("libcudart.so.13 { global: *; };\n")
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-std=c11", "-I/usr/local/cuda/include",
                    f"-Wl,--version-script={d / 'ver.map'}", "-Wl,-soname,libcudart.so.13",
                    "-o", str(d / "libcudart.so.13"), os.path.join(SIM, "cudart_shim.c")], check=True)
    return d


def _drive(shim_dir, names=()):
    env = dict(os.environ, LD_LIBRARY_PATH=str(shim_dir))
    r = subprocess.run([sys.executable, os.path.join(SIM, "drive.py"), *names], env=env, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    out = {}
    for line in r.stdout.splitlines():
        rec = json.loads(line)
        out[rec["case"]] = rec
    return out


@pytest.fixture(scope="module")
def records(shim_dir):
    return _drive(shim_dir)


@pytest.fixture(scope="module")
def full_records(shim_dir):
    import psutil
    if psutil.virtual_memory().available < 24 << 30:
        pytest.skip("the full-size host simulation maps about 20 GB of (untouched) buffers")
    return _drive(shim_dir, FULL_NAMES)


def _names(table):
    # the case lists, read from the driver's source without importing it (the
    # driver loads the library at import)
    src = open(os.path.join(SIM, "drive.py")).read()
    body = src.split(f"{table} = {{", 1)[1].split("\n}\n", 1)[0]
    return [line.split('"')[1] for line in body.splitlines() if line.strip().startswith('"')]


NAMES = _names("CASES")
FULL_NAMES = _names("FULL_CASES")


def test_every_case_ran(records):
    assert sorted(records) == sorted(NAMES)


@pytest.mark.parametrize("name", NAMES)
def test_case(records, name):
    _check(records[name])


def test_packed_factor_refused_before_device_work(shim_dir):
    """With JK_OPT_PACKED_FACTOR set, the adjoint, the dense-density calls, the
    host builds and their workspace queries return JK_ERR_UNSUPPORTED before
    any kernel, memset or copy."""
    rec = _drive(shim_dir, ["packed_refused"])["packed_refused"]
    assert rec["status"] == 0 and not rec["violations"], (rec["error"], rec["violations"])
    assert not rec["launches"] and rec["copies"] == 0


@pytest.mark.parametrize("name", FULL_NAMES)
def test_full_size_case(full_records, name):
    """The measured workloads at their full sizes (bench.py's shapes)."""
    _check(full_records[name])


def test_j_path_threshold_in_workspace_queries(shim_dir):
    """The split builds take J on the tensor cores above 4e9 multiply-adds of
    J's FP64 work: the queried workspace of the headline workload (automatic
    choice) equals that of the forced tensor-core form, the multi-state
    workload's that of the FP64 form, and nothing is launched."""
    rec = _drive(shim_dir, ["j_path_threshold"])["j_path_threshold"]
    assert rec["status"] == 0 and not rec["violations"], (rec["error"], rec["violations"])
    assert not rec["launches"]


def test_full_size_tuned_build_launch_count(full_records):
    """The tuned multi-state build (grouped schedule) issues 13 launches per
    build: grouped persistent GEMMs, grouped packing, exponent, slicer and
    reduction launches, the panel operands' row-wise exponent pass (a fill
    and a row launch), the FP64 metric dot and the FP64 J pass (at this size
    J's FP64 work, n(n+1)/2 naux nd = 1.5e9, is below the tensor-core
    threshold)."""
    assert len(full_records["full_multi_state_tuned"]["launches"]) == 13


def _check(rec):
    assert rec["status"] == 0, (rec["status"], rec["error"])
    assert rec["launches"], "no kernel was launched"
    for kname, grid, block, cluster, smem in rec["launches"]:
        assert 1 <= grid[0] <= 2**31 - 1 and 1 <= grid[1] <= 65535 and 1 <= grid[2] <= 65535, (kname, grid)
        assert 1 <= block[0] * block[1] * block[2] <= 1024, (kname, block)
        assert smem <= 227 * 1024, (kname, smem)
        assert cluster[0] * cluster[1] * cluster[2] <= 8 and grid[0] % cluster[0] == 0, (kname, grid, cluster)
    assert not rec["violations"], rec["violations"][:5]
    assert not rec["undecoded"] and rec["decoded"] == len(rec["launches"]), rec["undecoded"]
    owned = rec["owned"]
    for t in rec["tmaps"]:
        es = ESIZE[t["dtype"]]
        assert t["base"] % 16 == 0, t
        assert all(s % 16 == 0 and s < 2**40 for s in t["strides"][1:]), t
        assert all(1 <= b <= 256 for b in t["box"]), t
        inner = t["box"][0] * es
        assert inner % 16 == 0, t
        span = SWIZZLE_SPAN[t["swizzle"]]
        assert span is None or inner <= span, t
        lo = t["base"]
        hi = lo + t["dims"][0] * es + sum((dim - 1) * s for dim, s in zip(t["dims"][1:], t["strides"][1:]))
        inside = [o[2] for o in owned if o[0] <= lo and hi <= o[0] + o[1]]
        assert inside, f"tensor map [{lo:#x}, {hi:#x}) is outside every buffer of the call: {t}"


def _kernels(rec):
    return [k[0] for k in rec["launches"]]


@pytest.mark.parametrize("name,must", [
    ("dense_split", ["ozgemm_kernel", "frob_stream_kernel", "jstream_sym_kernel"]),
    ("dense_fp64", ["dgemm_nt_kernel", "frob_stream_kernel", "jstream_sym_kernel"]),
    ("grad_split_WV", ["ozgemm_kernel", "frob_stream_kernel", "axpy_kernel"]),
    ("pairs_split", ["ozgemm_kernel", "pair_dot_kernel"]),
    ("laplace_split", ["laplace_scale_kernel", "ozgemm_kernel"]),
    ("laplace_fp64_weighted", ["laplace_scale_kernel", "weighted_sum_kernel"]),
    ("build_split_fp32_digits", ["slice4f_kernel"]),
])
def test_expected_kernels(records, name, must):
    names = _kernels(records[name])
    for m in must:
        assert any(m in k for k in names), (m, sorted(set(names)))


def test_dense_split_needs_no_identity_panel(records):
    """K(D) reduces the panels against L itself: per aux chunk one panel GEMM
    for all densities and one reduction GEMM per density."""
    names = _kernels(records["dense_split"])
    assert sum("ozgemm_kernel" in k for k in names) == 1 + 2


# needs far less than the query, which covers both maps; no arena; skips what does not fit;
# packs its factor (no arena) before the build that runs out
FITS_IN_HALF = {"grad_fp64_V", "grad_fp64_V_packed", "noalloc", "autotune_split", "autotune_batched_split", "pack_factor_then_build"}


def test_too_small_arena_fails_before_any_device_work(shim_dir):
    """With half the queried arena every call reports JK_ERR_OOM and has
    enqueued nothing: no kernel, no memset, no copy."""
    recs = _drive(shim_dir, ["--arena-scale=0.5"])
    assert sorted(recs) == sorted(NAMES)
    for name, rec in recs.items():
        if name in FITS_IN_HALF:
            continue
        assert rec["status"] == 3 and ("arena" in rec["error"] or "workspace" in rec["error"]), (
            name, rec["status"], rec["error"])
        assert not rec["launches"] and rec["copies"] == 0, (name, len(rec["launches"]), rec["copies"])


def test_repeat_calls_are_capturable(shim_dir):
    """After one eager call on a handle, a second identical call creates no
    stream or event, sets no function attribute, looks nothing up and waits
    for nothing: the prerequisites for recording it in a CUDA graph.  (The
    autotuner times candidates and synchronizes by design.)"""
    recs = _drive(shim_dir, ["--twice"])
    assert sorted(recs) == sorted(NAMES)
    for name, rec in recs.items():
        assert rec["status"] == 0, (name, rec["error"])
        if name.startswith("autotune"):
            continue
        assert rec["syncs"] == 0 and rec["setups"] == 0, (name, rec["syncs"], rec["setups"])
        assert not rec["violations"], (name, rec["violations"][:3])


def test_library_imports_no_allocator():
    """libjk.so never allocates device or pinned memory: the CUDA runtime's
    allocation routines are not among its imports."""
    from paper_2608_06536_b300 import jk
    out = subprocess.run(["nm", "-D", "--undefined-only", jk.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    imported = {line.split()[-1].split("@")[0] for line in out.splitlines() if line.strip()}
    assert "cudaGetDevice" in imported
    banned = {s for s in imported if s.startswith("cuda") and ("Malloc" in s or "Free" in s or "HostAlloc" in s
                                                                or "HostRegister" in s)}
    assert not banned, banned


def test_random_cases(shim_dir):
    """Random entry points, shapes (tile and K-step edges, odd sizes) and
    options, under every per-call check above."""
    recs = _drive(shim_dir, ["--fuzz=200,7"])
    assert len(recs) == 200
    for name, rec in recs.items():
        try:
            _check(rec)
        except AssertionError as e:
            raise AssertionError(f"{name}: {e}") from None


def test_grouped_schedule_collapses_gemm_launches(full_records):
    """Launch collapse, counted on the CPU: the tuned multi-state build issues
    one sliced-GEMM launch for the panels of all densities and one for all
    eight rank updates; the per-density schedule (two aux chunks at this size)
    issues a panel launch and eight rank-update launches per chunk; J runs
    as the FP64 pass at this size (one launch for the grouped schedule)."""
    def gemms(name):
        return sum("ozgemm_kernel" in k[0] for k in full_records[name]["launches"])
    assert gemms("full_multi_state_tuned") == 2
    assert gemms("full_multi_state_default") == 2 * (1 + 8)
    assert sum("jstream_sym_kernel" in k[0] for k in full_records["full_multi_state_tuned"]["launches"]) == 1


def test_tuned_build_matches_the_measured_launch_list(full_records):
    """Kernel by kernel, the tuned multi-state build's launches: in the grouped
    schedule every operand of a wave is sliced by one slicer launch (the
    packed densities and the factor chunk after one exponent launch each,
    all densities' panel operands after the row-wise exponent pass over the
    panel) and every split-K reduction by one launch; gamma of the wave in
    one launch, J in one FP64 pass."""
    from collections import Counter
    per_build = {"ozgemm_kernel": 2, "expo_group_kernel": 2, "int_fill_kernel": 1, "panel_colmax_kernel": 1,
                 "slice_group_kernel": 3, "gamma_group_kernel": 1, "reduce_group_kernel": 1,
                 "pack_group_kernel": 1, "jstream_sym_kernel": 1}
    got = Counter()
    for k in full_records["full_multi_state_tuned"]["launches"]:
        got[next(key for key in per_build if key in k[0])] += 1
    assert dict(got) == per_build and sum(per_build.values()) == 13


EXEC_CASES = [n for n in NAMES if not n.startswith("autotune")]


def test_executed_calls_compute_the_oracle(shim_dir):
    """With each kernel's arithmetic executed at launch (numpy, on the memory
    standing in for the device's; the split GEMM as the exact product of its
    rebuilt 48-bit operands), every call of both engines, through the
    library's own host code, reproduces the oracle (the split paths to the
    48-bit rounding of their operands)."""
    recs = _drive(shim_dir, ["--exec", *EXEC_CASES])
    assert sorted(recs) == sorted(EXEC_CASES)
    for name, rec in recs.items():
        assert rec["status"] == 0 and rec["checks"], (name, rec["error"])
        worst = max(c[1] for c in rec["checks"])
        assert worst < 1e-12, (name, rec["checks"])


def test_random_executed_cases_compute_the_oracle(shim_dir):
    recs = _drive(shim_dir, ["--exec", "--fuzz=80,21"])
    checked = 0
    for name, rec in recs.items():
        assert rec["status"] == 0, (name, rec["error"])
        for label, err in rec["checks"]:
            assert err < 1e-12, (name, label, err)
            checked += 1
    assert checked > 40


REPEAT_EXEC = ["build_split", "build_fp64_chunks", "batched_split", "host_packed_split", "adjoint_split",
               "dense_split_chunks", "grad_split_WV", "pairs_split", "laplace_split", "noalloc"]


def test_repeat_calls_compute_the_oracle(shim_dir):
    """A second call on the same handle (arena, streams and flags left by the
    first) computes the oracle's values too."""
    recs = _drive(shim_dir, ["--exec", "--twice", *REPEAT_EXEC])
    for name in REPEAT_EXEC:
        rec = recs[name]
        assert rec["status"] == 0 and rec["checks"], (name, rec["error"])
        assert max(c[1] for c in rec["checks"]) < 1e-12, (name, rec["checks"])


FAULT_CASES = ["build_split", "build_split_grouped_raster1", "build_fp64_chunks", "batched_split",
               "host_packed_split", "adjoint_split", "dense_split_chunks", "grad_split_WV", "pairs_split",
               "laplace_split_weighted_sym", "noalloc"]


@pytest.mark.parametrize("at", [0, 1, 4])
def test_failed_launch_is_reported_and_the_handle_recovers(shim_dir, at):
    """A launch the runtime refuses (injected on the host) makes the call
    return JK_ERR_CUDA with a message naming the failure; an immediate retry
    on the same handle computes the oracle's values."""
    recs = _drive(shim_dir, ["--exec", f"--fail-launch={at}", *FAULT_CASES])
    for name in FAULT_CASES:
        rec = recs[name]
        first = rec["first"]
        assert first["status"] == 4, (name, first)
        if name != "noalloc":          # the arena-free build has no handle to hold a message
            assert "failed" in first["error"] and "/" not in first["error"], (name, first)
        assert rec["status"] == 0 and rec["checks"], (name, rec["error"])
        assert max(c[1] for c in rec["checks"]) < 1e-12, (name, rec["checks"])

"""The oracle (C), the host planner (C++) and the host blocked algorithm
(cpu_alg6, C++) built with AddressSanitizer and UndefinedBehaviorSanitizer and
run on the CPU (no GPU, no compute-sanitizer): every access and integer
operation of the oracle's entry points on small inputs, of the planner on
many chain shapes, modes and layouts, plus the public entry points on invalid
arguments and without a device (the device launchers are stand-ins that
report "no device"), and of the blocked algorithm on cut tiles, chains, in
place and several threads."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SAN = ["-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-fno-omit-frame-pointer", "-g", "-O1"]


def _cuda_home():
    nvcc = shutil.which("nvcc")
    home = os.environ.get("CUDA_HOME") or (os.path.dirname(os.path.dirname(nvcc)) if nvcc else "/usr/local/cuda")
    return home


def _run(exe):
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:] + r.stderr[-4000:]


@pytest.fixture(scope="module")
def gcc():
    if shutil.which("gcc") is None or shutil.which("g++") is None:
        pytest.skip("no gcc")
    return "gcc"


def test_oracle_under_asan_ubsan(tmp_path, gcc):
    exe = str(tmp_path / "oracle_san")
    cmd = ["gcc", *SAN, "-ffp-contract=off", "-std=c11",
           os.path.join(ROOT, "oracle", "spinsum_oracle.c"),
           os.path.join(ROOT, "tests", "sanitize", "oracle_driver.c"), "-o", exe, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("sanitizer runtime not available: " + r.stderr[-300:])
    assert r.returncode == 0, r.stderr
    _run(exe)


def test_host_planner_under_asan_ubsan(tmp_path, gcc):
    cuda = _cuda_home()
    inc = os.path.join(cuda, "include")
    libdir = next((p for p in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib")) if os.path.isdir(p)), None)
    if not os.path.exists(os.path.join(inc, "cuda_runtime.h")) or libdir is None:
        pytest.skip("CUDA runtime headers or library not found")
    exe = str(tmp_path / "host_san")
    csrc = os.path.join(ROOT, "paper_1705_06661_gb300", "csrc")
    cmd = ["g++", *SAN, "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", inc,
           os.path.join(csrc, "ss_host.cpp"),
           os.path.join(ROOT, "tests", "sanitize", "host_stubs.cpp"),
           os.path.join(ROOT, "tests", "sanitize", "host_driver.cpp"),
           "-o", exe, "-L", libdir, "-lcudart", f"-Wl,-rpath,{libdir}", "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("sanitizer runtime not available: " + r.stderr[-300:])
    assert r.returncode == 0, r.stderr[-4000:]
    _run(exe)


def test_host_alg6_under_asan_ubsan(tmp_path, gcc):
    exe = str(tmp_path / "alg6_san")
    cmd = ["g++", *SAN, "-ffp-contract=off", "-std=c++17", "-I", os.path.join(ROOT, "cpu_alg6"),
           os.path.join(ROOT, "cpu_alg6", "alg6.cpp"), os.path.join(ROOT, "cpu_alg6", "alg2.cpp"),
           os.path.join(ROOT, "tests", "sanitize", "alg6_driver.cpp"), "-o", exe, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("sanitizer runtime not available: " + r.stderr[-300:])
    assert r.returncode == 0, r.stderr
    _run(exe)


def test_threads_under_tsan(tmp_path, gcc):
    """The per-device lookup cache of the library and the host planner with
    its public entry points, called from many threads at once under
    ThreadSanitizer (device launchers stubbed)."""
    cuda = _cuda_home()
    inc = os.path.join(cuda, "include")
    libdir = next((p for p in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib")) if os.path.isdir(p)), None)
    if not os.path.exists(os.path.join(inc, "cuda_runtime.h")) or libdir is None:
        pytest.skip("CUDA runtime headers or library not found")
    exe = str(tmp_path / "thread_san")
    csrc = os.path.join(ROOT, "paper_1705_06661_gb300", "csrc")
    cmd = ["g++", "-fsanitize=thread", "-g", "-O1", "-std=c++17", "-I", os.path.join(ROOT, "include"), "-I", inc,
           os.path.join(csrc, "ss_host.cpp"),
           os.path.join(ROOT, "tests", "sanitize", "host_stubs.cpp"),
           os.path.join(ROOT, "tests", "sanitize", "thread_driver.cpp"),
           "-o", exe, "-L", libdir, "-lcudart", f"-Wl,-rpath,{libdir}", "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("sanitizer runtime not available: " + r.stderr[-300:])
    assert r.returncode == 0, r.stderr[-4000:]
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=1:second_deadlock_stack=1")
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout[-2000:] + r.stderr[-4000:]
    assert "WARNING: ThreadSanitizer" not in r.stderr, r.stderr[-4000:]

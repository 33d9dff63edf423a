"""Host sanitizers: the oracle and the C ABI's host code under AddressSanitizer
and UndefinedBehaviorSanitizer.

Each test reruns existing CPU test files in a child pytest that starts with
libasan preloaded and loads the instrumented build (liboracle_asan.so,
libvdbc_asan.so).  Both builds stop at the first report
(-fno-sanitize-recover=all), so any out-of-bounds access, use after free,
signed overflow, bad shift or misaligned load fails the child."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


def asan_runtime():
    try:
        p = subprocess.run(["gcc", "-print-file-name=libasan.so"], stdout=subprocess.PIPE, text=True).stdout.strip()
    except OSError:
        p = ""
    if not os.path.isabs(p) or not os.path.exists(p):
        pytest.skip("no libasan for this gcc")
    return p


def child_env(extra):
    e = dict(os.environ)
    e.update(extra)
    e["LD_PRELOAD"] = asan_runtime()
    e["ASAN_OPTIONS"] = "detect_leaks=0:abort_on_error=1"
    e["UBSAN_OPTIONS"] = "print_stacktrace=1:halt_on_error=1"
    e["PYTHONPATH"] = ROOT + os.pathsep + e.get("PYTHONPATH", "")
    return e


def run_pytest(files, extra_env, timeout=900):
    env = child_env(extra_env)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "not gpu"] +
                       [os.path.join(HERE, f) for f in files], cwd=ROOT, env=env, stdout=subprocess.PIPE,
                       stderr=subprocess.STDOUT, text=True, timeout=timeout)
    out = r.stdout
    assert r.returncode == 0, out[-6000:]
    assert "AddressSanitizer" not in out and "runtime error" not in out, out[-6000:]
    return out


def loaded_library(module, extra_env):
    code = "import %s as m; print(getattr(m, 'LIB_PATH', None) or m.LIB)" % module
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=child_env(extra_env), stdout=subprocess.PIPE,
                       stderr=subprocess.STDOUT, text=True, timeout=300)
    assert r.returncode == 0, r.stdout
    return r.stdout.strip().splitlines()[-1]


def prebuild(code, extra_env):
    """Builds an instrumented library in a process without libasan preloaded
    (the compilers themselves must not run under it)."""
    e = dict(os.environ)
    e.update(extra_env)
    e["PYTHONPATH"] = ROOT + os.pathsep + e.get("PYTHONPATH", "")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=e, stdout=subprocess.PIPE,
                       stderr=subprocess.STDOUT, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-4000:]


def test_oracle_under_asan_and_ubsan():
    """Every oracle pin (encoder, codecs, renderer, network) on the
    instrumented oracle."""
    env = {"ORACLE_SANITIZE": "1"}
    prebuild("import oracle; oracle.build()", env)
    assert loaded_library("oracle", env).endswith("liboracle_asan.so")
    files = sorted(f for f in os.listdir(HERE) if f.startswith("test_oracle_") and f.endswith(".py"))
    assert len(files) >= 4
    out = run_pytest(files, env)
    assert " passed" in out


def test_c_abi_host_code_under_asan_and_ubsan():
    """The C ABI's host paths that run without a device (argument checks,
    error strings, grid-file parsing and validation) on the instrumented
    library."""
    env = {"VDBC_SANITIZE": "1"}
    prebuild("from paper_2504_04564_gb300 import build; build.build(sanitize=True); build.build(checked=True)", {})
    assert loaded_library("paper_2504_04564_gb300", env).endswith("libvdbc_asan.so")
    out = run_pytest(["test_abi.py"], env)
    assert " passed" in out

"""The host side of the C-ABI (argument checks, workspace layout and sizes)
under AddressSanitizer and UndefinedBehaviorSanitizer: the library is built
with both on its host code and the host ABI tests (and the layout property
tests) run against it in a child process; any sanitizer report fails the
test.  No GPU is used."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _runtime(name):
    cc = shutil.which("gcc")
    if not cc:
        return None
    path = subprocess.run([cc, f"-print-file-name={name}"], capture_output=True, text=True).stdout.strip()
    return path if os.path.isabs(path) and os.path.exists(path) else None


def test_host_abi_under_sanitizers(tmp_path):
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not (asan and ubsan):
        pytest.skip("gcc's sanitizer runtimes are not installed")
    from paper_2510_03312_gb300 import build as B
    B.build()  # the regular library, which the host tests' fixture expects to be current
    lib = B.build_sanitized(str(tmp_path / "san"))
    code = (
        "import sys, pytest\n"
        f"sys.path.insert(0, {ROOT!r}); sys.path.insert(0, {os.path.join(ROOT, 'tests')!r})\n"
        "from paper_2510_03312_gb300 import ubs as U\n"
        f"U.load({lib!r})\n"
        f"sys.exit(pytest.main(['-q', '-p', 'no:cacheprovider', {os.path.join(ROOT, 'tests', 'test_abi_host.py')!r}, "
        f"{os.path.join(ROOT, 'tests', 'test_abi_layout_props.py')!r}]))\n"
    )
    env = dict(os.environ, LD_PRELOAD=f"{asan} {ubsan}", ASAN_OPTIONS="detect_leaks=0:halt_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=600)
    out = r.stdout + r.stderr
    assert "AddressSanitizer" not in out and "runtime error" not in out, out[-4000:]
    assert r.returncode == 0, out[-4000:]
    assert " passed" in out

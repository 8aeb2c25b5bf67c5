"""The bounds-checking build (-DCG_BOUNDS_CHECK, libchordal_debug.so): on the
CPU, the error-word description and the release build's refusal to inject;
on a GPU (marked), the dense, batched, CSR and sweep parity suites run
against the bounds-checking build in a child process (every launch is then
checked and any out-of-range index would fail its call with CG_ECUDA), and
an injected error travels from the device error word to CG_ECUDA."""
import ctypes
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1508_06329_gb300 import build, binding
    build.build()
    return binding.load()


def describe(word: int) -> str:
    from paper_1508_06329_gb300 import binding as B
    buf = ctypes.create_string_buffer(256)
    assert B.cg_debug_describe(ctypes.c_uint64(word), buf, 256) == B.CG_OK
    return buf.value.decode()


def test_error_word_description(lib):
    assert describe(0) == "no bounds-check error"
    assert describe((1 << 56) | 70000) == "dense LexBFS cls index 70000 out of range"
    assert describe((16 << 56) | 5) == "CSR LexBFS cls index 5 out of range"
    assert describe((255 << 56) | 0) == "injected test entry index 0 out of range"
    assert "unknown array" in describe((200 << 56) | 1)


def test_release_build_refuses_injection(lib):
    from paper_1508_06329_gb300 import binding as B
    if b"bounds-checking" in B.cg_version():
        pytest.skip("this process loaded the bounds-checking build")
    assert B.cg_debug_inject(255) == B.CG_EINVAL
    assert b"not a bounds-checking build" in B.cg_last_error_string()
    assert B.cg_debug_inject(0) == B.CG_EINVAL


INJECT = r"""
import numpy as np, torch
import graphgen as gg, oracle
from paper_1508_06329_gb300 import binding as B
assert b"bounds-checking" in B.cg_version(), B.cg_version()
g = gg.subtree_dense(500, 80, 1)
rows = torch.from_numpy(np.ascontiguousarray(g.rows).view(np.int32)).cuda()
res = torch.empty(4, dtype=torch.int32, device="cuda")
with B.Context(0) as ctx:
    assert B.cg_debug_inject(255) == B.CG_OK
    try:
        B.chordal_test_dense(ctx, rows, g.n, res)
        raise SystemExit("no error reported")
    except B.ChordalError as e:
        assert e.status == B.CG_ECUDA and "injected test entry" in str(e), str(e)
    B.chordal_test_dense(ctx, rows, g.n, res)      # the word was cleared: the next call is clean
    torch.cuda.synchronize()
    assert tuple(res.cpu().tolist()) == oracle.chordal_test(g).witness
print("inject ok")
"""


@pytest.mark.gpu
def test_parity_suites_under_the_bounds_checking_build():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1508_06329_gb300 import build
    debug_lib = build.build(debug=True)
    env = dict(os.environ, CG_LIBCHORDAL=debug_lib)
    r = subprocess.run([sys.executable, "-c", INJECT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "inject ok" in r.stdout, r.stdout + r.stderr
    skip = ("full_size or large_pair or batch_workload_full or step_floor or sweep_large or plus_chain_large "
            "or cta_sizes")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider", "-m", "gpu",
                        "tests/test_gpu_dense.py", "tests/test_gpu_batch.py", "tests/test_gpu_csr.py",
                        "tests/test_gpu_sweep.py", "-k", "not (" + skip + ")"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert " passed" in r.stdout and " failed" not in r.stdout

import os
import subprocess
import sys
import tempfile
import time

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (runs through the C-ABI library)")
    config.addinivalue_line("markers", "slow: long-running CPU check")
    config.addinivalue_line("markers", "fullsize(cfg): whole solve of a full-size configuration against the "
                                       "oracle's whole solve (minutes of host-core work)")


# Whole oracle solves of the full-size configurations run in one subprocess, started
# as soon as the selected tests are known (before any test touches the GPU), so
# that their host-core minutes overlap the other GPU tests.
_FULLSIZE = {"proc": None, "dir": None, "names": []}


def _start_fullsize(names):
    if _FULLSIZE["proc"] is not None or not names:
        return
    import oracle
    oracle.build()   # before the subprocess imports it
    d = tempfile.mkdtemp(prefix="vi_fullsize_")
    log = open(os.path.join(d, "oracle.log"), "w")
    _FULLSIZE["proc"] = subprocess.Popen([sys.executable, os.path.join(HERE, "fullsize_oracle.py"), d] + names,
                                         stdout=log, stderr=subprocess.STDOUT)
    _FULLSIZE["dir"] = d
    _FULLSIZE["names"] = list(names)


def pytest_collection_finish(session):
    names = []
    for item in session.items:
        m = item.get_closest_marker("fullsize")
        if m and m.args and m.args[0] not in names:
            names.append(m.args[0])
    if not names:
        return
    try:
        import torch
        if not torch.cuda.is_available():
            return
    except Exception:
        return
    # the largest first: the tests wait for them in the same order
    order = {"cfg4": 0, "cfg2": 1, "cfg3": 2}
    _start_fullsize(sorted(names, key=lambda n: order.get(n, 9)))


@pytest.fixture(scope="session")
def fullsize_oracle():
    """Returns a function name -> dict(V, policy, iters, seconds, cores) that waits for
    the subprocess's result of that configuration."""
    def get(name, timeout_s=3600.0):
        if _FULLSIZE["proc"] is None:
            _start_fullsize([name])
        d = _FULLSIZE["dir"]
        path, err = os.path.join(d, f"{name}.npz"), os.path.join(d, f"{name}.err")
        t0 = time.time()
        while not os.path.exists(path):
            if os.path.exists(err):
                raise RuntimeError(open(err).read())
            if _FULLSIZE["proc"].poll() is not None and not os.path.exists(path):
                raise RuntimeError("oracle subprocess ended without a result for " + name + ": " +
                                   open(os.path.join(d, "oracle.log")).read()[-2000:])
            if time.time() - t0 > timeout_s:
                raise TimeoutError(f"oracle solve of {name} not done after {timeout_s:.0f} s")
            time.sleep(2.0)
        z = np.load(path)
        return {k: z[k] for k in z.files}
    yield get
    p = _FULLSIZE["proc"]
    if p is not None and p.poll() is None:
        p.terminate()
        try:
            p.wait(timeout=10)
        except subprocess.TimeoutExpired:
            p.kill()


@pytest.fixture(scope="session", autouse=True)
def _built_libraries():
    """Compile the oracle and the CUDA library in-tree if they are missing (nvcc
    cross-compiles for sm_103a without a GPU)."""
    import oracle
    oracle.build()
    from paper_2303_10672_b300 import build as cuda_build
    cuda_build.build()
    yield

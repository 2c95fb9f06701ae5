import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running (full-size sampled parity)")
    _ensure_host_libs()


def _ensure_host_libs():
    """Compile the generator and the oracle if this checkout has not built them yet."""
    for src, out in (("gen/sinet_gen.c", "gen/_lib/libsinet_gen.so"),
                     ("oracle/sinet_oracle.c", "oracle/_lib/liboracle.so")):
        src_p, out_p = os.path.join(ROOT, src), os.path.join(ROOT, out)
        if os.path.exists(out_p) and os.path.getmtime(out_p) >= os.path.getmtime(src_p):
            continue
        os.makedirs(os.path.dirname(out_p), exist_ok=True)
        subprocess.run(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11", src_p, "-o",
                        out_p + ".tmp", "-lm"], check=True)
        os.replace(out_p + ".tmp", out_p)


@pytest.fixture(scope="session")
def orc():
    import oracle

    return oracle.get()

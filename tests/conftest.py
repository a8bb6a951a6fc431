import os
import sys
from pathlib import Path

# The oracle's sparse LU and BLAS calls run single-threaded: predictable
# timings, no oversubscription when tests run beside other CPU work.
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import pytest

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the library's kernels)")
    config.addinivalue_line("markers", "slow: takes tens of seconds on a CPU")


@pytest.fixture(scope="session")
def fe():
    """The C-ABI binding with the library built for sm_103a."""
    from paper_0704_2344_gb300 import build, fe as fe_mod
    build.build()
    fe_mod.load()
    return fe_mod


@pytest.fixture(scope="session")
def ctx(fe):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test without a CUDA device: run these with -m gpu on a GPU machine")
    torch.cuda.init()
    stream = torch.cuda.Stream()
    c = fe.fe_ctx_create(0, stream=stream.cuda_stream)
    c.torch_stream = stream
    yield c
    fe.fe_ctx_synchronize(c)
    fe.fe_ctx_destroy(c)

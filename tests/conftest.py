import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def load_golden(name):
    """Parse a tests/golden/*.txt fixture into {section: [[float]]} plus m, n."""
    path = os.path.join(ROOT, "tests", "golden", name)
    out, cur = {}, None
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("m "):
                parts = line.split()
                out["m"], out["n"] = int(parts[1]), int(parts[3])
                continue
            if line.replace("_", "").isalnum() and not line[0].isdigit() and not line[0] == "-":
                cur = line
                out[cur] = []
                continue
            out[cur].append([float(v) for v in line.split()])
    return out


def loo_gate(variant, n, kappa, loo_oracle):
    """Loss-of-orthogonality gate of a GPU result.  The O(u) variants meet the
    FP64 gate 1e-12; BCGSI+1s has O(u) kappa^2 loss of orthogonality (Table 1),
    so it is held to that bound with a modest constant and to at most ten
    times the oracle's own loss of orthogonality on the same input."""
    if variant != "bcgsi+1s":
        return 1e-12
    u = 2.0 ** -53
    return min(10 * n * u * kappa ** 2, max(1e-12, 10 * loo_oracle))


@pytest.fixture
def golden():
    return load_golden


def ensure_library():
    """Build libbcgs_qr.so in-tree if it is missing (nvcc cross-compiles without a GPU)."""
    lib = os.path.join(ROOT, "paper_2507_21791_gb300", "libbcgs_qr.so")
    if not os.path.exists(lib):
        import __graft_entry__

        __graft_entry__.build()
    return lib


@pytest.fixture(scope="session")
def cuda():
    """The CUDA path: skips without a GPU, builds the library if needed."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_library()
    from paper_2507_21791_gb300 import bcgs

    bcgs.load_library()
    return bcgs

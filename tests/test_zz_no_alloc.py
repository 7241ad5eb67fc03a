"""The allocation-free coarsest solve, dcg_coarse_solve_static, against the
allocating entry point dcg_coarse_solve on the same inputs.

Some callers cannot allocate device memory where they need the solve (their
device memory is already reserved by a caching allocator, or they run a
latency-critical loop that must not take an allocation's implicit
synchronisation); the static variant keeps its scratch in a fixed array
inside the library instead. The file name makes pytest collect it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mg
from paper_2606_13429_gb300 import dcg, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2606_13429_gb300 import build
    build.build()
    dcg.load()
    torch.cuda.set_device(0)


def _coarse_nodes(d, n, levels):
    return (mg.level_sizes(n, levels)[-1] - 1) ** d


# m + 1 a power of two (sine transforms by FFT: 8, 128, 16) and not (dense
# passes with the sine matrix: 48, 12), so both routes use the static scratch
@pytest.mark.parametrize("d,n,levels", [(2, 64, 4), (2, 256, 2), (3, 32, 2), (2, 96, 2), (3, 24, 2)])
def test_static_matches_allocating_twice(d, n, levels):
    prob = dcg.dcg_assemble(d, n, 1e-3)
    dcg.dcg_setup(prob, dcg.options(max_levels=levels))  # FP64 cycle
    nn = _coarse_nodes(d, n, levels)
    assert prob.level_nodes(1) == nn
    for call in range(2):  # the shared scratch keeps the previous call's contents
        f = torch.from_numpy(inputs.rhs(30 + call, nn)).cuda()
        z_ref = torch.empty_like(f)
        dcg.dcg_coarse_solve(prob, f, z_ref)
        z = torch.full_like(f, float("nan"))
        dcg.dcg_coarse_solve_static(prob, f, z)
        torch.cuda.synchronize()
        a, b = z.cpu().numpy(), z_ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(b)


def test_static_rejects_coarse_levels_above_the_limit():
    prob = dcg.dcg_assemble(2, 768, 1e-3)
    dcg.dcg_setup(prob, dcg.options(max_levels=2))  # coarsest 383^2 = 146,689 nodes
    nn = _coarse_nodes(2, 768, 2)
    assert nn > 131072
    f = torch.zeros(nn, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(f)
    with pytest.raises(dcg.DCGError) as err:
        dcg.dcg_coarse_solve_static(prob, f, z)
    assert err.value.code == dcg.DCG_ERR_INVALID_ARG
    assert "DCG_STATIC_COARSE_MAX" in str(err.value)

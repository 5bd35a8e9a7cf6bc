"""The energy entry point that allocates nothing (hho_energy_static).

Some callers cannot allocate device memory when they want the energy check:
for instance a hook between time steps in a framework whose caching
allocator owns the device memory, or code with a fixed memory budget
(cudaFree would also synchronise the device).  hho_energy_static keeps its
scratch in a fixed array inside the library.  This test calls it through the
C ABI twice in a row and compares each result with hho_energy, which uses a
caller-provided work buffer.  It lives in its own file, collected last, and
passes alone in a fresh process as well as after the other tests.
"""
import numpy as np
import pytest

import synth
from tests.libutil import ensure_built

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    from paper_2505_15771_gb300 import hho, solver
    return hho, solver


def test_energy_static_matches_energy_twice(lib):
    hho, solver = lib
    md = synth.hybrid_grid(24, 20, 0.0, 1.0, 0.0, 1.0, 0.7, 0.5)
    P = solver.Problem(md, synth.layered_media(md), 2)
    out = torch.full((2,), float("nan"), dtype=torch.float64, device=P.dev)
    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((3, 4)):
        x = P.to_device(synth.random_state(P.layout.n_canonical, seed))
        ref = P.energy(x)                               # hho_energy with a caller work buffer
        hho.hho_energy_static(P.ops, x.data_ptr(), out[call:].data_ptr(), stream)
        got = float(out[call].item())
        assert np.isfinite(got)
        assert abs(got - ref) <= 1e-12 * abs(ref), (call, got, ref)
    assert float(out[0].item()) != float(out[1].item())
    P.close()


def test_energy_static_rejects_null_arguments(lib):
    hho, solver = lib
    assert hho.lib().hho_energy_static(None, None, None, None) == hho.HHO_EINVAL

"""The split-BF16 tcgen05 products (tensor cores, FP32 accumulation in
tensor memory) against FP64 products of the same operands."""
import numpy as np
import pytest

from tests.libutil import ensure_built

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hho():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return ensure_built()


@pytest.mark.parametrize("K,N", [(16, 16), (32, 32), (64, 48), (48, 128)])
def test_split_bf16_gemm(hho, K, N):
    """Each operand is hi + lo in BF16 (16 significant bits); the dropped
    lo lo product and the FP32 accumulation leave an error of a few 2^-16
    of sum_k |a_k b_k|.  A distinct value in every entry catches any
    transposed or misplaced operand tile."""
    rng = np.random.default_rng(K * 1000 + N)
    A = rng.standard_normal((128, K)).astype(np.float32)
    B = rng.standard_normal((K, N)).astype(np.float32)
    D, status = hho.hho_tc_gemm_check(A, B)
    assert status == 0
    ref = A.astype(np.float64) @ B.astype(np.float64)
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64)
    err = np.abs(D - ref) / scale
    print("K=%d N=%d: max |D - AB| / (|A||B|) = %.3e (2^-16 = %.3e)" % (K, N, err.max(), 2.0 ** -16))
    assert err.max() <= 4 * 2.0 ** -16
    # a single-term BF16 product would be far worse: the split is in effect
    assert err.max() <= 0.05 * np.abs(A.astype(np.float64)) .max() * 2.0 ** -8 * K or err.max() < 2.0 ** -14


MESHES = [
    ("quad_k2", lambda: __import__("synth").quad_grid(8, 6, 0.0, 1.2, 0.0, 1.0, 0.5), 2),
    ("hybrid_k3", lambda: __import__("synth").hybrid_grid(8, 8, 0.0, 1.0, 0.0, 1.0, 0.7, 0.5), 3),
    ("tri_k1", lambda: __import__("synth").tri_grid(8, 8), 1),
    ("hanging_k2", lambda: __import__("synth").hanging_node_patch(8, 6, refine_rows=(2, 3)), 2),
    ("basin_k2", lambda: __import__("synth").basin_c5(nx=40, ny=10)["mesh"], 2),
]


@pytest.mark.parametrize("name,make,k", MESHES, ids=[m[0] for m in MESHES])
@pytest.mark.parametrize("shots", [1, 3, 16, 64])
def test_bf16x3_stage_against_fp64(hho, name, make, k, shots):
    """The tensor-core batched stage (HHO_BF16X3) against the FP64 batched
    path (which equals the oracle shot by shot) after 20 ERK4 steps from
    seeded random states with one point force per shot: every shot's state
    within 1e-4 relative L2, the error flag clear, and the same order of
    error as the FP32 path (split BF16 keeps 16 significant bits of each
    operand, FP32 24)."""
    import synth
    from paper_2505_15771_gb300 import solver
    md = make()
    media = synth.layered_media(md)
    P = solver.Problem(md, media, k)
    try:
        rng = np.random.default_rng(shots + k)
        lo, hi = md.xy.min(axis=0), md.xy.max(axis=0)
        pts = [tuple(lo + (0.15 + 0.7 * rng.random(2)) * (hi - lo)) for _ in range(shots)]
        P.set_shot_sources(pts, [(0.0, 1.0)] * shots, 10.0)
        n = P.layout.n_canonical
        U0 = np.stack([synth.random_state(n, 70 + i) for i in range(shots)])
        dt = (0.004 if name != "basin_k2" else 0.0004) / k
        out = {}
        for prec in (hho.HHO_F64, hho.HHO_F32, hho.HHO_BF16X3):
            x = P.batch_to_device(U0, prec)
            _, work = P.batch_buffers(4, shots, prec)
            P.batch_step(x, work, shots, 4, 0.0, dt, 20, precision=prec)
            out[prec] = P.batch_to_canonical(x, shots, prec)
        assert hho.hho_tc_error(P.ops) == 0
    finally:
        P.close()
    ref = out[hho.HHO_F64]
    e32 = max(np.linalg.norm(out[hho.HHO_F32][i] - ref[i]) / np.linalg.norm(ref[i]) for i in range(shots))
    etc = max(np.linalg.norm(out[hho.HHO_BF16X3][i] - ref[i]) / np.linalg.norm(ref[i]) for i in range(shots))
    print("%s k=%d shots=%d: rel L2 vs FP64, FP32 %.2e, split-BF16 tensor cores %.2e" % (name, k, shots, e32, etc))
    assert etc <= 1e-4
    assert etc <= 200 * max(e32, 1e-8)

"""The packed GEMM path (tcgen05 TF32 / 3xTF32 / BF16x3, float64 SIMT) against numpy float64."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

# bound on max|C - C_ref| / (max|A| max|B| K) for each precision mode; the shapes cover
# ragged M/N/K tails, several tiles, split-K (long K, few tiles) and grouped rasterisation
TOL = {0: 1e-15, 1: 2e-3, 2: 2e-6, 3: 3e-5}
# tensor-core tiles forced through RTCC_GEMM_TILE ("" = the planner's own choice): every kernel
# instantiation (N = 64, 128, 256; every variant of the wider two) runs each case
TILES = ["", "256:0", "256:1", "256:2", "128:0", "128:1", "128:2", "64:0"]


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("shape", [(1, 8, 8, 4), (2, 300, 200, 77), (1, 129, 257, 130), (3, 64, 40, 1000), (2, 40, 30, 6000), (1, 1100, 700, 300)])
def test_gemm_matches_float64(prec, shape, tile, monkeypatch):
    from paper_2205_05175_gb300 import rtcc
    if tile and prec == 0:
        pytest.skip("the float64 path has no tensor-core tile")
    if tile:
        monkeypatch.setenv("RTCC_GEMM_TILE", tile)
    nb, M, N, K = shape
    rng = np.random.default_rng(1234 + M)
    A = rng.standard_normal((nb, M, K))
    B = rng.standard_normal((nb, N, K))
    ref = np.einsum("bmk,bnk->bmn", A, B)
    C = rtcc.rtcc_selftest_gemm(prec, A, B)
    err = np.abs(C - ref).max() / (np.abs(A).max() * np.abs(B).max() * K)
    assert err < TOL[prec], err
    # the tensor-core modes must not be exact (they run in reduced precision on the tensor cores)
    if prec in (1, 3) and K > 8:
        assert np.abs(C - ref).max() > 0


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("prec", [0, 1, 2, 3])
@pytest.mark.parametrize("kinds", ["cr", "rc", "cc"])
@pytest.mark.parametrize("shape", [(2, 150, 70, 90), (1, 33, 300, 1200), (3, 300, 130, 40), (1, 1000, 50, 200)])
def test_complex_gemm_matches_float64(prec, kinds, shape, tile, monkeypatch):
    """Complex operands: re/im planes and the segment table (Ar Br - Ai Bi, Ar Bi + Ai Br).
    Short K loops take the both-planes work items (ragged 128-wide and 64-wide tiles)."""
    from paper_2205_05175_gb300 import rtcc
    if tile and prec == 0:
        pytest.skip("the float64 path has no tensor-core tile")
    if tile:
        monkeypatch.setenv("RTCC_GEMM_TILE", tile)
    nb, M, N, K = shape
    rng = np.random.default_rng(99 + N)
    A = rng.standard_normal((nb, M, K)) + (1j * rng.standard_normal((nb, M, K)) if kinds[0] == "c" else 0)
    B = rng.standard_normal((nb, N, K)) + (1j * rng.standard_normal((nb, N, K)) if kinds[1] == "c" else 0)
    ref = np.einsum("bmk,bnk->bmn", A, B)
    C = rtcc.rtcc_selftest_gemm(prec, A, B)
    err = np.abs(C - ref).max() / (np.abs(A).max() * np.abs(B).max() * K)
    assert err < 2 * TOL[prec], err


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("prec", [2, 3])
@pytest.mark.parametrize("kinds", ["rr", "cc"])
def test_long_k_accumulation_is_chunked(prec, kinds, tile, monkeypatch):
    """A long K loop of same-sign products (K = 32768, nonnegative inputs, so the sum grows with
    every product): the split modes accumulate on the tensor cores in chunks of 16 K blocks summed
    with round-to-nearest float32 adds, which holds the result to a few parts in 10^6 of itself.
    The allocation-free entry point keeps one float32 accumulation over the whole K loop; its error
    is printed beside (the drift that chunking removes).  Every tile instantiation is forced in
    turn (RTCC_GEMM_TILE), so each chunk-fold protocol (sum in TMEM with one or two slots, sum in
    the epilogue's registers) runs."""
    import torch
    if tile:
        monkeypatch.setenv("RTCC_GEMM_TILE", tile)

    from paper_2205_05175_gb300 import rtcc
    nb, M, N, K = 1, 128, 96, 32768
    rng = np.random.default_rng(5)
    A = rng.random((nb, M, K)) + (1j * rng.random((nb, M, K)) if kinds == "cc" else 0)
    B = rng.random((nb, N, K)) + (1j * rng.random((nb, N, K)) if kinds == "cc" else 0)
    ref = np.einsum("bmk,bnk->bmn", A, B)
    C = rtcc.rtcc_selftest_gemm(prec, A, B)
    err = np.abs(C - ref).max() / np.abs(ref).max()
    tc = torch.zeros((nb, M, N), dtype=torch.complex128 if kinds == "cc" else torch.float64, device="cuda")
    try:
        rtcc.rtcc_gemm_noalloc(prec, torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), tc)
        torch.cuda.synchronize()
        err_one = f"{np.abs(tc.cpu().numpy() - ref).max() / np.abs(ref).max():.2e}"
    except rtcc.RtccError:      # packed operands beyond the entry point's static scratch
        err_one = "n/a"
    print(f"prec {prec} {kinds}: chunked {err:.2e}, one accumulation {err_one}")
    assert err < 1e-5, (err, err_one)


@pytest.mark.parametrize("tile", TILES)
@pytest.mark.parametrize("shape", [(40, 128, 256, 3000), (60, 64, 300, 2000), (24, 200, 260, 5000), (9, 130, 257, 8100)])
def test_chunked_split_k_items(shape, tile, monkeypatch):
    """Long K over few output tiles: the K loop is split across CTAs, and with chunked accumulation
    (BF16x3) items of one or two chunks and short remainders follow each other on one CTA, the
    case in which the single-sum protocol must not run a phase ahead of the epilogue.  Every tile
    instantiation is forced in turn."""
    from paper_2205_05175_gb300 import rtcc
    if tile:
        monkeypatch.setenv("RTCC_GEMM_TILE", tile)
    nb, M, N, K = shape
    rng = np.random.default_rng(4321 + K)
    A = rng.standard_normal((nb, M, K))
    B = rng.standard_normal((nb, N, K))
    ref = np.einsum("bmk,bnk->bmn", A, B)
    for _ in range(3):
        C = rtcc.rtcc_selftest_gemm(3, A, B)
        err = np.abs(C - ref).max() / (np.abs(A).max() * np.abs(B).max() * K)
        assert err < TOL[3], err

"""The tile-shape autotuner of the sliced block products (negf_tune_products,
negf_set_product_variant, paper_2602_03438_gb300.tuning): every variant gives the
product of the definition, the tuner picks a variant that supports the block size, and
a saved tuning loads into another context unchanged."""
import json

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-13   # the sliced product's bound relative to the row x column norms


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_03438_gb300 as P
    P.negf.load_library()
    return P


@pytest.mark.parametrize("n,variants", [(48, (1, 2, 3)), (100, (1, 2, 3)), (128, (1, 2, 3)), (200, (3,))])
def test_every_variant_gives_the_product(P, n, variants):
    ctx = P.Context(0, 1 << 30)
    try:
        rng = np.random.default_rng(n)
        U = 37
        A = rng.normal(size=(U, n, n)) + 1j * rng.normal(size=(U, n, n))
        B = rng.normal(size=(U, n, n)) + 1j * rng.normal(size=(U, n, n))
        A *= 10.0 ** rng.uniform(-4, 4, size=(1, n, 1))     # rows of very different scales
        exact = A @ B
        size = np.linalg.norm(A, axis=2)[:, :, None] * np.linalg.norm(B, axis=1)[:, None, :]
        tA, tB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        for v in (0,) + tuple(variants):
            ctx.check(ctx.lib.negf_set_product_variant(ctx.h, n, v))
            D = torch.empty_like(tA)
            P.negf.negf_block_gemm(ctx, P.MIXED, tA, tB, D)
            assert ctx.sync() == 0
            assert (np.abs(D.cpu().numpy() - exact) / size).max() <= TOL, v
        for v in (1, 2):
            if v not in variants:
                assert ctx.lib.negf_set_product_variant(ctx.h, n, v) == P.negf.NEGF_ERR_ARG
    finally:
        ctx.close()


def test_tuner_choices_round_trip_through_json(P, tmp_path):
    ctx = P.Context(0, 2 << 30)
    ctx2 = P.Context(0, 64 << 20)
    try:
        path = str(tmp_path / "tuning.json")
        res = P.tuning.tune(ctx, [32, 96, 128, 192, 8], units=128, path=path)
        ch = res["choices"]
        assert ch["8"]["variant"] == 0 and ch["8"]["ms"] == {}        # no sliced product below n = 16
        for n in ("32", "96", "128"):
            assert ch[n]["variant"] in (1, 2, 3) and set(ch[n]["ms"]) == {"1", "2", "3"}
            assert ch[n]["ms"][str(ch[n]["variant"])] == min(ch[n]["ms"].values())
        assert ch["192"]["variant"] == 3 and set(ch["192"]["ms"]) == {"3"}
        saved = P.tuning.load(ctx2, path)
        assert saved == json.load(open(path))
    finally:
        ctx.close()
        ctx2.close()

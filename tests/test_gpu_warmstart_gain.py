"""What the trained warm-start network gains over the method without it.

The full pipeline on the GPU: training pairs from the plain solver (decimation +
Newton polishing, FP64), the network trained by the library's own kernels, and the
guess-driven OBC on held-out energies, compared with (a) the plain decimation and
(b) the same guess-driven solver started from a zero guess (the method without the
network: its first Newton step from zero is g = a00^{-1}).

Two regimes, reported with eta and the numbers (printed; run with -s to see them):
  * the warm-start workload as stated (b = 64 leads, eta = 1e-6): Newton's basin for
    the surface equation is about eta wide in the propagating channels, so guesses
    with the network's held-out error are not kept; the plain solver stays the fallback
    and every energy still converges;
  * a broadened, smaller lead (b = 8, eta = 5e-2), where the network's guesses are
    inside the basin: the network removes most decimation steps, which a zero guess
    does not.  Time is reported, not asserted: each Newton step sums a Stein series
    by Smith doubling, so fewer decimation steps do not mean less time.
"""
import json

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2602_03438_gb300 as P
    P.negf.load_library()
    return P


def _run(P, b, eta, steps, lr=3e-4):
    from paper_2602_03438_gb300 import warmstart as WS
    sets = W.config5_sets(b=b)
    H00, H01 = sets["H00"], sets["H01"]
    ctx = P.Context(0, 4 << 30)
    try:
        lt, Et = sets["train"]
        tr = WS.solve_surfaces(ctx, WS.lead_system(H00, H01, lt, Et, eta))
        # the few energies whose residual stalls just above 1e-10 (NEGF_ERR_NOCONV) still
        # give targets accurate far beyond the network's error; they stay in the set
        noconv = int((tr.status != 0).sum())
        assert noconv <= len(lt) // 100
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        X = P.negf.negf_mlp_pack(ctx, b, t(H00), t(H01), t(lt), t(Et))
        net = WS.train_network(ctx, b, X, tr.gs_R.contiguous(), len(lt), W.mlp_init(b, 512), steps=steps,
                               batch=256, lr=lr)
        lh, Eh = sets["held"]
        sh = WS.lead_system(H00, H01, lh, Eh, eta)
        cold = WS.solve_surfaces(ctx, sh)
        g0, ms_net = WS.predict(ctx, net, H00, H01, lh, Eh)
        warm = WS.solve_surfaces(ctx, sh, g0_R=g0)
        zero = WS.solve_surfaces(ctx, sh, g0_R=torch.zeros_like(g0))
        ref = cold.gs_R
        err = lambda g: (torch.linalg.matrix_norm(g - ref) / torch.linalg.matrix_norm(ref)).cpu().numpy()
        kept_w, kept_z = warm.iters[:, 1] == 0, zero.iters[:, 1] == 0
        out = dict(
            b=b, eta=eta, train_pairs=len(lt), train_noconv=noconv, held_out=len(lh), train_steps=steps,
            loss_first_last=[net.losses[0][1], net.losses[-1][1]],
            guess_err_median=float(np.median(err(g0))),
            plain=dict(decimation_steps=float(cold.iters[:, 1].mean()), newton=float(cold.newton[:, 1].mean()),
                       ms=cold.ms),
            network=dict(kept=float(kept_w.mean()), decimation_steps=float(warm.iters[:, 1].mean()),
                         newton=float(warm.newton[:, 1].mean()), ms=warm.ms + ms_net, ms_network=ms_net),
            zero_guess=dict(kept=float(kept_z.mean()), decimation_steps=float(zero.iters[:, 1].mean()),
                            newton=float(zero.newton[:, 1].mean()), ms=zero.ms),
        )
        print(json.dumps(out))
        # the plain solver is the arbiter: every energy converged, whichever path it took,
        # to the same retarded surface function
        for r in (cold, warm, zero):
            assert np.all(r.status == 0) or np.array_equal(r.status != 0, cold.status != 0)
        ok = cold.status == 0
        assert err(warm.gs_R)[ok].max() <= 1e-9 and err(zero.gs_R)[ok].max() <= 1e-9
        return out
    finally:
        ctx.close()


def test_gain_on_the_stated_workload(P):
    # Measured: the held-out guess error stays ~1 (g(E) of a 64-orbital lead at eta =
    # 1e-6 varies on scales far below the 0.023 spacing of the training energies), no
    # guess is kept, and the failed Newton attempts add time.  What is asserted is that
    # the OBC stays correct with the network in the loop (inside _run).
    out = _run(P, 64, 1e-6, steps=2000)
    assert out["network"]["decimation_steps"] == out["plain"]["decimation_steps"] or out["network"]["kept"] > 0


def test_gain_where_the_guess_is_inside_the_basin(P):
    out = _run(P, 8, 5e-2, steps=4000)
    assert out["guess_err_median"] < 0.3
    assert out["network"]["kept"] > 0.5 > out["zero_guess"]["kept"]
    assert out["network"]["decimation_steps"] < 0.5 * out["plain"]["decimation_steps"]

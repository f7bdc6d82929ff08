"""CPU-only checks of the C ABI: the library loads, exports every entry point
declared in include/negf.h, and its integer batch layout is bit-exact."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in ("negf.h", "negf_warmstart.h")]


@pytest.fixture(scope="module")
def lib():
    from paper_2602_03438_gb300 import negf
    if not os.path.exists(negf.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return negf.load_library()


def declared_functions():
    txt = "".join(open(h).read() for h in HEADERS)
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(negf_[a-z_]+)\s*\(", txt)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    for n in ["negf_obc", "negf_rgf_retarded", "negf_rgf_lesser", "negf_observables", "negf_ctx_create"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2602_03438_gb300 import negf
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(negf.EXPORTS) <= set(declared_functions())


def _layout_py(shapes):
    """Exclusive prefix sums of the packing, recomputed in Python."""
    acc = [0] * 8
    rows = []
    for nb, b, ne in shapes:
        rows.append(list(acc))
        bb = b * b
        inc = [nb * bb, (nb - 1) * bb, ne, ne * bb, ne * nb * bb, ne * (nb - 1) * bb, ne * (nb - 1), nb * b]
        acc = [a + i for a, i in zip(acc, inc)]
    rows.append(acc)
    return np.array(rows, dtype=np.int64)


def test_uneven_layout_is_bit_exact(lib):
    from paper_2602_03438_gb300 import negf
    shapes = W.config3_shapes()
    assert len(shapes) == 256
    got = negf.system_layout([s[0] for s in shapes], [s[1] for s in shapes], [s[2] for s in shapes])
    assert np.array_equal(got, _layout_py(shapes))
    # every (device, energy, block) addressed exactly once
    tot = got[-1]
    assert tot[4] == sum(ne * nb * b * b for nb, b, ne in shapes)


def test_layout_rejects_bad_shapes(lib):
    from paper_2602_03438_gb300 import negf
    with pytest.raises(negf.NegfError) as ei:
        negf.system_layout([4], [513], [2])
    assert ei.value.code == negf.NEGF_ERR_ARG
    with pytest.raises(negf.NegfError):
        negf.system_layout([0], [8], [2])


def test_null_arguments_are_rejected_without_a_gpu(lib):
    from paper_2602_03438_gb300 import negf
    assert lib.negf_obc(None, None, 0, 1e-12, 10, None, None, None, None, None, None, None, None, None,
                        None) == negf.NEGF_ERR_ARG
    assert lib.negf_rgf_lesser(None, None, 0, None, None, None, None, None, None, None, None, None,
                               None, None, None) == negf.NEGF_ERR_ARG
    assert lib.negf_layout(None, None) == negf.NEGF_ERR_ARG
    assert b"NULL" in lib.negf_last_error(None)


def test_mlp_dims_match_the_oracle_layout(lib):
    from paper_2602_03438_gb300 import negf
    from oracle import mlp_oracle as M
    for b, h in ((64, 512), (8, 128), (16, 256)):
        d = negf.negf_mlp_get_dims(b, h)
        k0, k0p, hid, nout = M.mlp_dims(b, h)
        lay, total = M.param_layout(b, h)
        assert (d.b, d.hidden, d.k0, d.k0p, d.nout) == (b, h, k0, k0p, nout)
        assert [d.off_W1, d.off_c1, d.off_W2, d.off_c2, d.off_W3, d.off_c3] == [lay[k][0] for k in
                                                                             ("W1", "c1", "W2", "c2", "W3", "c3")]
        assert d.n_params == total
        assert negf.negf_mlp_workspace_bytes(d, 1000) > negf.negf_mlp_workspace_bytes(d, 100) > 0
    for b, h in ((12, 512), (64, 100), (0, 512)):
        with pytest.raises(negf.NegfError) as ei:
            negf.negf_mlp_get_dims(b, h)
        assert ei.value.code == negf.NEGF_ERR_ARG


def test_mlp_entry_points_reject_null_without_a_gpu(lib):
    from paper_2602_03438_gb300 import negf
    assert lib.negf_mlp_pack(None, 64, 1, 1, None, None, None, None, None, None) == negf.NEGF_ERR_ARG
    assert lib.negf_mlp_forward(None, None, None, 1, None, None, None) == negf.NEGF_ERR_ARG
    assert lib.negf_mlp_train_step(None, None, None, None, None, None, 1, 1e-3, 1, None, 0, None, None, None, 1,
                                   None) == negf.NEGF_ERR_ARG


def _worklist_py(shapes, block_size):
    """The (device, energy) units of the devices with one block size, in device-then-
    energy order, with their output offsets, recomputed in Python from the layout."""
    L = _layout_py(shapes)
    units = dict(unit_dev=[], unit_e=[], off_d=[], off_o=[])
    for d, (nb, b, ne) in enumerate(shapes):
        if b != block_size or ne == 0:
            continue
        for e in range(ne):
            units["unit_dev"].append(d)
            units["unit_e"].append(e)
            units["off_d"].append(L[d][4] + e * nb * b * b)
            units["off_o"].append(L[d][5] + e * (nb - 1) * b * b)
    return {k: np.array(v, dtype=np.int64) for k, v in units.items()}


def test_uneven_batch_worklist_is_bit_exact(lib):
    """The work list of the batched sweeps over config 3's 256 devices (every block size),
    and of a batch with empty devices, against a Python recomputation."""
    from paper_2602_03438_gb300 import negf
    shapes = W.config3_shapes()
    cases = [shapes, [(3, 16, 4), (5, 8, 0), (2, 16, 3), (4, 24, 5), (1, 16, 2)]]
    for sh in cases:
        nb, bs, ne = zip(*sh)
        for b in sorted(set(bs)):
            got = negf.system_worklist(nb, bs, ne, b)
            ref = _worklist_py(sh, b)
            assert got["unit_dev"].size == ref["unit_dev"].size
            for k in ref:
                assert np.array_equal(got[k].astype(np.int64), ref[k]), (b, k)
    # a block size no device has: no units
    assert negf.system_worklist([3], [16], [4], 32)["unit_dev"].size == 0

"""The C-ABI library builds, loads without a GPU and exports every entry
point that include/fabric.h declares (no compute calls)."""
import ctypes
import os

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def lib():
    from paper_2406_17782_gb300 import build
    build.build()
    import paper_2406_17782_gb300 as pkg
    return pkg.load()


def test_every_declared_symbol_is_exported(lib):
    import paper_2406_17782_gb300 as pkg
    names = pkg.header_functions()
    assert "fabric_shade_reference" in names and "fabric_train_step" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_the_four_calls_of_the_path_are_declared():
    import paper_2406_17782_gb300 as pkg
    names = set(pkg.header_functions())
    for n in ("fabric_encode_params", "fabric_shade_reference", "fabric_shade_neural", "fabric_train_step"):
        assert n in names


def test_struct_layouts_match_header(lib):
    from paper_2406_17782_gb300._abi import FabricGBuffer, FabricMaterial, FabricTrainBatch
    assert ctypes.sizeof(FabricMaterial) == 84 == W.MATERIAL_DTYPE.itemsize
    assert ctypes.sizeof(FabricGBuffer) == 7 * 8
    assert ctypes.sizeof(FabricTrainBatch) == 8 * 8
    # field offsets of the numpy record equal the C struct's
    for name, off in [("pattern", 0), ("twist_deg", 4), ("incl_deg", 8), ("alpha", 12), ("beta", 20),
                      ("kd", 28), ("ks", 52), ("gap", 76), ("w_blend", 80)]:
        assert W.MATERIAL_DTYPE.fields[name][1] == off


def test_param_counts(lib):
    import oracle
    assert lib.fabric_decoder_param_count() == oracle.mlp.n_params(oracle.mlp.DEC_SHAPES) == 13188
    assert lib.fabric_encoder_param_count() == oracle.mlp.n_params(oracle.mlp.ENC_SHAPES) == 23584
    assert len(W.decoder_init()) == 13188 and len(W.encoder_init()) == 23584


def test_paper_structure_param_counts(lib):
    """The library's layout of the paper decoder and its two ablations
    equals the oracle's (and the initialisers'), at both widths; unknown
    widths and structures give -1."""
    from oracle import mlp as M
    from oracle import paper_net as PN
    from paper_2406_17782_gb300._abi import PAPER_STRUCTURES
    abl = {"full": PN.FULL, "no_oneblob": PN.NO_ONEBLOB, "no_fusion": PN.NO_FUSION}
    for w in PN.WIDTHS:
        assert lib.fabric_paper_param_count(w, 0) == lib.fabric_paper_structure_param_count(w, 0)
        for name, a in PAPER_STRUCTURES.items():
            n = M.n_params(PN.dec_shapes(w, abl[name]))
            assert lib.fabric_paper_structure_param_count(w, a) == n == len(W.paper_decoder_init(w, ablation=name))
    # S1 [64][67] (no one-blob) has 21 * 64 fewer weights; without fusion
    # the first layer [W][93] and A1 [W][W] hold as many as S1 [W][88] and
    # A1 [W][W+5]
    assert lib.fabric_paper_structure_param_count(64, 1) == lib.fabric_paper_structure_param_count(64, 0) - 21 * 64
    assert lib.fabric_paper_structure_param_count(64, 2) == 27076
    assert lib.fabric_paper_structure_param_count(128, 2) == lib.fabric_paper_structure_param_count(128, 0)
    assert lib.fabric_paper_structure_param_count(96, 0) == -1
    assert lib.fabric_paper_structure_param_count(64, 3) == -1


def test_status_strings_and_null_context(lib):
    assert lib.fabric_status_string(0) == b"FABRIC_OK"
    assert lib.fabric_status_string(6) == b"FABRIC_ERR_UNSUPPORTED"
    # calls on a NULL context are rejected on the host, before any CUDA call
    assert lib.fabric_set_materials(None, None, 0) == 1
    assert lib.fabric_shade_reference(None, None, 1, 1, 0, None, None, None) == 1
    assert lib.fabric_sync_status(None, None) == 1


def test_no_oracle_in_product_path():
    """The product package never imports or links the oracle."""
    pkg_dir = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2406_17782_gb300")
    for root, _, files in os.walk(pkg_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cpp")):
                text = open(os.path.join(root, f)).read()
                assert "import oracle" not in text and "from oracle" not in text and "liboracle" not in text, f

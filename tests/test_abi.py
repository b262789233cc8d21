"""The C-ABI library builds, loads without a GPU, and exports every call the header declares."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "blindmatch.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bm_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_protocol_calls():
    names = declared_functions()
    for call in ["bm_keygen", "bm_encode_gallery", "bm_encrypt_query", "bm_match", "bm_decrypt_scores"]:
        assert call in names


def test_library_exports_every_declared_symbol():
    from paper_2408_06167_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol():
    from paper_2408_06167_gb300 import binding
    missing = [n for n in declared_functions() if not hasattr(binding, n) and n not in binding._SIGS]
    assert not missing, missing


def test_presets_and_errors_without_gpu():
    from paper_2408_06167_gb300 import binding as bm
    p = bm.bm_params_preset("ring16")
    assert (p.log_n, p.n_q, p.n_p, p.dnum, p.secret_hw) == (16, 4, 2, 2, 192)
    assert list(p.q_bits[:4]) == [60, 40, 40, 40] and list(p.p_bits[:2]) == [60, 60]
    try:
        bm.bm_params_preset(7)
    except bm.BlindMatchError as e:
        assert e.status == 1
    else:
        raise AssertionError("unknown preset accepted")


def test_context_refuses_shapes_outside_the_kernels():
    """The key-switching, rescale and NTT kernels cover rings 2^12 and 2^16, digits
    of at most two primes and at most two special primes; other parameter sets are
    refused before any device work (so this runs without a GPU)."""
    from paper_2408_06167_gb300 import binding as bm
    cases = []
    for log_n in (11, 13, 14, 15, 17):
        p = bm.bm_params_preset("small4")
        p.log_n = log_n
        cases.append(p)
    p = bm.bm_params_preset("small4")
    p.n_p, p.p_bits[2] = 3, 60
    cases.append(p)
    p = bm.bm_params_preset("small4")
    p.dnum = 1                       # one digit of four primes
    cases.append(p)
    for p in cases:
        try:
            bm.bm_context_create(p)
        except bm.BlindMatchError as e:
            assert e.status == 2, (p.log_n, p.n_p, p.dnum, str(e))
        else:
            raise AssertionError(f"accepted log_n={p.log_n} n_p={p.n_p} dnum={p.dnum}")

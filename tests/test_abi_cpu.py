"""CPU-only checks of the C ABI: the library builds for sm_103a, loads, and
exports every entry point that include/rpcg.h declares (no GPU calls)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(rpcg_[a-z0-9_]+)\s*\(", src))
    return names


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("rpcg_create", "rpcg_destroy", "rpcg_dot_exact", "rpcg_dot_fpe", "rpcg_solve"):
        assert required in names


def _declarations_with_comments():
    """(name, the comment block that documents it) for every function the
    header declares: the block right before it, or before the group of
    declarations it belongs to."""
    out = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        tokens = re.finditer(r"/\*.*?\*/|\b(?:rpcg_status|void|const char \*)\s*(rpcg_[a-z0-9_]+)\s*\([^;]*;", src, flags=re.S)
        last_comment = None
        for m in tokens:
            if m.group(0).startswith("/*"):
                last_comment = m.group(0)
            else:
                out.append((m.group(1), last_comment))
    return out


def test_every_declaration_is_documented_and_cites_the_paper():
    decls = _declarations_with_comments()
    assert {n for n, _ in decls} == declared_symbols()
    for name, comment in decls:
        assert comment, name
    # the compute entry points cite the passage that defines their operation
    cites = re.compile(r"Sec\. \d|Alg\. \d|Fig\. \d|Listing \d")
    for name, comment in decls:
        if name in ("rpcg_spmv", "rpcg_dot_exact", "rpcg_dot_fpe", "rpcg_solve", "rpcg_batch_solve",
                    "rpcg_create", "rpcg_eft_twosum", "rpcg_eft_twoprod"):
            assert cites.search(comment), name


def test_library_exports_every_declared_symbol(rpcg):
    L = ctypes.CDLL(rpcg.LIB_PATH)
    missing = [n for n in sorted(declared_symbols()) if not hasattr(L, n)]
    assert not missing, missing
    assert sorted(declared_symbols()) == sorted(set(rpcg.EXPORTS) | (declared_symbols() - set(rpcg.EXPORTS)))


def test_status_strings_and_defaults(rpcg):
    L = rpcg.lib()
    assert L.rpcg_status_string(0) == b"ok"
    assert L.rpcg_status_string(-2).startswith(b"matrix not SPD")
    o = rpcg.Opts()
    L.rpcg_opts_default(ctypes.byref(o))
    assert o.tol == 1e-8 and o.max_iter == 1000 and o.fpe_size == 8 and o.fpe_strict == 0


def test_invalid_arguments_rejected_without_gpu(rpcg):
    L = rpcg.lib()
    # argument checks happen before any CUDA call
    assert L.rpcg_dot_exact(-1, None, None, None, None) == rpcg.ERR_INVALID
    assert L.rpcg_dot_exact(10, None, None, ctypes.c_void_p(8), None) == rpcg.ERR_INVALID
    assert L.rpcg_dot_fpe(4, ctypes.c_void_p(8), ctypes.c_void_p(8), 9, ctypes.c_void_p(8), ctypes.c_void_p(8),
                          None) == rpcg.ERR_INVALID
    assert b"p must be" in L.rpcg_last_error()
    h = ctypes.c_void_p()
    rp = (ctypes.c_int32 * 3)(0, 1, 5)  # rowptr[n] != nnz
    assert L.rpcg_create(ctypes.byref(h), 2, 2, rp, rp, rp, 0, None) == rpcg.ERR_INVALID
    # rows beyond the documented limit (32-bit index headroom), before any array is read
    assert L.rpcg_create(ctypes.byref(h), 2 ** 31 - 1, 0, None, None, None, 0, None) == rpcg.ERR_INVALID
    assert b"at most" in L.rpcg_last_error()


def test_library_has_no_cpu_fallback_symbols(rpcg):
    """The product path is the CUDA library only; it never links the oracle."""
    import subprocess
    out = subprocess.run(["nm", "-D", rpcg.LIB_PATH], capture_output=True, text=True).stdout
    assert "oracle_" not in out

"""C-ABI library: builds, loads without a GPU and exports every declared
symbol; host-side argument checks run without touching the device."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "airga.h")


@pytest.fixture(scope="module")
def G():
    from paper_1606_01216_gb300 import build
    build.build()
    from paper_1606_01216_gb300 import airga
    airga.lib()
    return airga


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(airga_[a-z0-9_]+)\s*\(", text)))


def test_header_declarations_are_exported(G):
    decl = declared_functions()
    assert len(decl) >= 20
    L = G.lib()
    for name in decl:
        assert hasattr(L, name), name
    assert sorted(G.EXPORTS) == decl


def test_no_torch_or_cuda_types_in_header():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    for bad in ("torch", "at::", "cudaStream_t", "#include <cuda"):
        assert bad not in text


def test_host_only_calls(G):
    assert G.lib().airga_version() == 100
    o = G.options()
    assert o.tol == 1e-10 and o.maxit == 20000 and o.pattern_hbw == 3 and o.symmetrize == 1
    assert o.mr_tol == 0.01 and o.mr_kmax == 50 and o.spai_mode == G.SPAI_QR
    assert o.inner_tol == 3e-4 and o.max_outer == 12 and o.mr_relative == 0
    assert o.want_colres == 1 and o.sm_share == 1 and o.reserved0 == 0
    assert G.status_string(G.E_UNSUPPORTED).startswith("operation not available")
    assert G.status_string(1234) == "unknown status"


def test_header_is_plain_c(tmp_path):
    """include/airga.h compiles as strict C99 (no C++ or CUDA types leak in)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    src = tmp_path / "use_header.c"
    src.write_text('#include "airga.h"\n'
                   "int main(void) { airga_options o; airga_trace_record r; (void)o; (void)r;\n"
                   "  return 0; }\n")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", inc,
                        "-c", str(src), "-o", str(tmp_path / "use_header.o")],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_trace_host_side(G):
    """Tracing state is host-side: enabling, reading an empty trace and
    turning it off need no GPU; bad arguments are rejected."""
    G.trace_enable(8)
    try:
        recs, dropped = G.trace_read()
        assert recs == [] and dropped == 0
        with pytest.raises(G.AirgaError):
            G.trace_enable(-1)
        n = C.c_int32()
        assert G.lib().airga_trace_read(None, -1, C.byref(n), None) == G.E_INVALID_ARG
        assert G.lib().airga_trace_read(None, 4, C.byref(n), None) == G.E_INVALID_ARG
        assert G.lib().airga_trace_read(None, 0, C.byref(n), None) == G.OK and n.value == 0
    finally:
        G.trace_enable(0)


def test_argument_checks_need_no_gpu(G):
    L = G.lib()
    out = C.c_void_p()
    # n < 1 and NULL arrays are rejected before any CUDA call
    assert L.airga_mat_from_csr(0, 0, None, None, None, None, C.byref(out)) == G.E_INVALID_ARG
    assert "n must be" in G.last_error()
    assert L.airga_mat_from_csr(5, 3, None, None, None, None, C.byref(out)) == G.E_INVALID_ARG
    assert L.airga_assemble_shifted(None, None, 0.1, 1e-4, 1.0, None, C.byref(out)) == G.E_INVALID_ARG
    assert L.airga_spai_build(None, None, None, None, C.byref(out)) == G.E_INVALID_ARG
    assert L.airga_mat_to_csr(None, None, None, None, None) == G.E_INVALID_ARG
    assert L.airga_mat_is_banded(None) == 0 and L.airga_mat_nnz(None) == 0
    assert L.airga_precond_factor_nnz(None, 0) == 0 and L.airga_precond_is_banded(None) == 0
    assert L.airga_precond_factor_csr(None, 0, None, None, None, None) == G.E_INVALID_ARG
    assert L.airga_precond_from_csr(0, 1, None, None, None, None, None, C.byref(out)) \
        == G.E_INVALID_ARG
    assert L.airga_spai_update(None, None, None, None, None, C.byref(out)) == G.E_INVALID_ARG
    assert L.airga_pcg_solve(None, None, None, 1, None, None, None, None, None, None, None) \
        == G.E_INVALID_ARG
    assert L.airga_precond_length(None) == 0 and L.airga_mat_rows(None) == 0
    assert L.airga_debug_set_fault(99) == G.E_INVALID_ARG
    assert L.airga_debug_set_fault(G.FAULT_NONE) == G.OK
    assert L.airga_precond_from_bands(10, 0, None, None, C.byref(out)) == G.E_INVALID_ARG
    L.airga_mat_free(None)
    L.airga_precond_free(None)


def test_options_layout_matches_header(G):
    # offsets follow C's natural alignment of the struct in airga.h
    O = G.Options
    assert O.tol.offset == 0 and O.maxit.offset == 8 and O.mr_tol.offset == 16
    assert O.barrier_timeout_ms.offset == 40 and O.want_colres.offset == 44
    assert O.inner_tol.offset == 48
    assert O.max_outer.offset == 56 and O.mr_relative.offset == 60
    assert O.sm_share.offset == 64 and C.sizeof(O) == 72


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, "paper_1606_01216_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "airga_oracle" not in text and "liboracle" not in text, f


def test_mlp_options_layout_and_defaults(G):
    O = G.MlpTrainOptions
    assert O.lr.offset == 0 and O.beta1.offset == 4 and O.beta2.offset == 8 and O.eps.offset == 12
    assert O.batch.offset == 16 and O.cosine_steps.offset == 20 and O.seed.offset == 24
    assert C.sizeof(O) == 32
    o = G.mlp_train_options()
    assert o.batch == 4096 and o.cosine_steps == 0 and abs(o.lr - 2e-3) < 1e-9
    assert abs(o.beta1 - 0.9) < 1e-7 and abs(o.beta2 - 0.999) < 1e-7 and o.eps > 0


def test_mlp_argument_checks_need_no_gpu(G):
    L = G.lib()
    out = C.c_void_p()
    assert L.airga_mlp_spai(None, None, 1.0, 0.1, 1e-4, None, C.byref(out)) == G.E_INVALID_ARG
    assert L.airga_mlp_grad(None, None, None, None, 10, None, 4, None, None, None) == G.E_INVALID_ARG
    assert L.airga_mlp_train(None, None, None, None, 10, 1, None, None, None, None) == G.E_INVALID_ARG
    assert L.airga_mlp_forward(None, None, 1, None, None) == G.E_INVALID_ARG
    assert L.airga_mlp_features(None, None, 1.0, 0.1, 1e-4, None, 1, None, None, None, None,
                                None) == G.E_INVALID_ARG
    assert L.airga_mlp_set_params(None, None, None) == G.E_INVALID_ARG
    assert L.airga_mlp_spai(None, None, 1.0, 0.1, 1e-4, None, None) == G.E_INVALID_ARG
    L.airga_mlp_free(None)

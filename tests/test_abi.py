"""CPU checks of the C-ABI library: it builds for sm_103a, loads without a GPU,
and exports every function include/ie.h declares; the binding's struct layouts
match the header's field lists."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ie.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ie_[A-Za-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2310_18043_gb300 import build as b
    path = b.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    fns = declared_functions()
    for f in ["ie_create", "ie_filter_apply", "ie_solve", "ie_destroy", "ie_status_str",
              "ie_apply_G", "ie_hsrr", "ie_spmv", "ie_get_coeffs", "ie_get_factor",
              "ie_get_stats", "ie_opts_default"]:
        assert f in fns


def test_library_exports_every_declared_symbol(lib):
    for f in declared_functions():
        assert hasattr(lib, f), f"{f} not exported"


def test_binding_knows_every_export():
    import paper_2310_18043_gb300.ie as ie
    assert sorted(ie.EXPORTS) == declared_functions()


def test_struct_layouts_match_header():
    import paper_2310_18043_gb300.ie as ie
    src = open(HEADER).read()

    src_nc = re.sub(r"/\*.*?\*/", "", src, flags=re.S)

    def fields(name):
        body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + ";", src_nc).group(1)
        out = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            for piece in decl.split(","):
                out.append(re.findall(r"[A-Za-z_]\w*", piece)[-1])
        return out

    assert [f for f, _ in ie.ie_opts._fields_] == fields("ie_opts")
    assert [f for f, _ in ie.ie_stats._fields_] == fields("ie_stats")
    assert [f for f, _ in ie.ie_pencil._fields_] == fields("ie_pencil")
    assert [f for f, _ in ie.ie_batch_item._fields_] == fields("ie_batch_item")


def test_struct_offsets_match_c_compiler(tmp_path):
    """sizeof and every field offset of the ABI structs, as gcc lays them out from the
    header, equal the binding's ctypes layout."""
    import shutil
    import subprocess
    import paper_2310_18043_gb300.ie as ie
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"ie_opts": ie.ie_opts, "ie_stats": ie.ie_stats, "ie_pencil": ie.ie_pencil,
               "ie_batch_item": ie.ie_batch_item, "ie_complex": ie.ie_complex}
    lines = ["#include <stdio.h>", "#include <stddef.h>", f'#include "{HEADER}"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'  printf("{name} %zu\\n", sizeof({name}));')
        for f, _ in cls._fields_:
            lines.append(f'  printf("{name}.{f} %zu\\n", offsetof({name}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-o", str(exe), str(src)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], check=True,
               capture_output=True, text=True).stdout.splitlines())
    for name, cls in structs.items():
        assert int(got[name]) == ctypes.sizeof(cls), name
        for f, _ in cls._fields_:
            assert int(got[f"{name}.{f}"]) == getattr(cls, f).offset, (name, f)


def test_status_strings_and_defaults(lib):
    import paper_2310_18043_gb300.ie as ie
    assert ie.ie_status_str(ie.IE_OK) == "IE_OK"
    assert "NOCONV" in ie.ie_status_str(ie.IE_ERR_NOCONV)
    o = ie.ie_opts_default()
    assert (o.k, o.driver, o.m_max, o.max_outer) == (16, 1, 100, 10)
    assert (o.tau_g, o.tau, o.gmres_tol, o.sigma_is_center) == (1e-2, 1e-10, 1e-12, 1)
    assert (o.precision, o.refine_steps, o.adjoint) == (0, 8, 0)


def test_argument_checks_need_no_gpu(lib):
    """Entry points reject invalid arguments before any CUDA call, so these run on a host
    without a GPU: a NULL handle, an empty batch."""
    import paper_2310_18043_gb300.ie as ie
    assert ie.ie_destroy(None) == ie.IE_ERR_ARG
    st, _ = ie.ie_solve_batch([])
    assert st == ie.IE_ERR_ARG
    assert ie.load().ie_solve_batch(None, 3, 0) == ie.IE_ERR_ARG


def test_no_oracle_in_product_path():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2310_18043_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f


def test_block_marshalling_reads_column_major_layouts():
    """The binding passes a block as (pointer, leading dimension, rows, columns) and accepts
    only column-major complex128 blocks (numpy Fortran order or a transposed torch tensor)."""
    import numpy as np
    import paper_2310_18043_gb300.ie as ie
    a = np.zeros((10, 3), dtype=np.complex128, order="F")
    p, ld, n, k = ie._block(a)
    assert (ld, n, k) == (10, 10, 3) and p.value == a.ctypes.data
    big = np.zeros((13, 3), dtype=np.complex128, order="F")
    p, ld, n, k = ie._block(big[:10])                     # ragged leading dimension
    assert (ld, n, k) == (13, 10, 3)
    with pytest.raises(ValueError):
        ie._block(np.zeros((10, 3), dtype=np.complex128))  # row-major
    with pytest.raises(TypeError):
        ie._block(np.zeros((10, 3), dtype=np.complex64, order="F"))
    torch = pytest.importorskip("torch")
    t = torch.zeros((3, 10), dtype=torch.complex128).T     # n x k view of a (k, n) tensor
    p, ld, n, k = ie._block(t)
    assert (ld, n, k) == (10, 10, 3)


def test_binding_rejects_output_blocks_of_the_wrong_shape():
    """The library writes n x k outputs through raw pointers, with k and the leading
    dimension taken from the input block. The binding refuses, before any library call, an
    output narrower or shorter than the input, a 1-D output for k > 1, and blocks whose row
    count differs from the handle's n."""
    import numpy as np
    import paper_2310_18043_gb300.ie as ie
    h = 0x5EED                                    # a handle value the binding has seen created
    ie._handle_n[h] = 10
    try:
        V = np.zeros((10, 3), dtype=np.complex128, order="F")
        for bad in (np.zeros((10, 2), dtype=np.complex128, order="F"),
                    np.zeros(10, dtype=np.complex128),
                    np.zeros((9, 3), dtype=np.complex128, order="F")):
            for fn in (ie.ie_apply_G, ie.ie_apply_G_static, ie.ie_apply_GH, ie.ie_filter_apply):
                with pytest.raises(ValueError):
                    fn(h, V, bad)
            with pytest.raises(ValueError):
                ie.ie_spmv(h, 0, V, bad)
        short = np.zeros((11, 3), dtype=np.complex128, order="F")
        with pytest.raises(ValueError):
            ie.ie_apply_G(h, short, short)        # rows differ from the handle's n
        with pytest.raises(ValueError):
            ie.ie_hsrr(h, V, np.zeros((10, 2), dtype=np.complex128, order="F"))
        with pytest.raises(ValueError):
            ie.ie_solve(h, None, np.zeros((10, 2), dtype=np.complex128, order="F"), 3)
        with pytest.raises(ValueError):
            ie.ie_solve_left(h, np.ones(3), np.zeros((10, 2), dtype=np.complex128, order="F"))
        with pytest.raises(ValueError):
            ie.ie_eig_sensitivity(h, V, V, 1j, None, np.ones(3), np.zeros(9))
    finally:
        ie._handle_n.pop(h, None)

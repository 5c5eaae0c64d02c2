"""The C-ABI library loads and exports every entry point include/glasso.h declares; its
argument checks answer without touching a GPU.  CPU only."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "glasso.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(glasso_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("glasso_create", "glasso_destroy", "glasso_solve", "glasso_solve_batch",
                     "glasso_submit", "glasso_poll", "glasso_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(glasso):
    lib = C.CDLL(glasso.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_declared()) == set(glasso.EXPORTED)


def test_status_strings_and_defaults(glasso):
    assert glasso.glasso_status_string(0) == b"GLASSO_OK"
    assert glasso.glasso_status_string(10) == b"GLASSO_LINESEARCH_STALL"
    cfg = glasso.glasso_config()
    assert glasso.glasso_config_default(C.byref(cfg)) == 0
    assert cfg.max_iter == 500 and cfg.shrink == 0.5 and cfg.t_min == 1e-4 and cfg.precision == 0
    assert cfg.products == glasso.PRODUCTS["auto"] == 0
    # the binding's structures match the header's layout
    assert C.sizeof(glasso.glasso_profile) == 3 * 8 * len(glasso.PROF_CLASSES)


def test_bad_products_option_is_rejected(glasso):
    cfg = glasso.glasso_config()
    glasso.glasso_config_default(C.byref(cfg))
    cfg.products = 7
    h = C.c_void_p()
    assert glasso.glasso_create(C.byref(cfg), C.byref(h)) == 1  # GLASSO_ERR_ARG, before any CUDA call
    assert not h.value


def test_argument_checks_need_no_gpu(glasso):
    # NULL handle / NULL outputs are rejected before any CUDA call
    assert glasso.glasso_create(None, None) == 1
    assert glasso.glasso_solve(None, None, 0, 0, 10, 0.1, 1e-6, None, None, None) == 1
    assert glasso.glasso_destroy(None) == 0
    assert glasso.glasso_last_error(None) == b""


def test_create_without_a_gpu_is_refused_cleanly(glasso):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    cfg = glasso.glasso_config()
    glasso.glasso_config_default(C.byref(cfg))
    h = C.c_void_p()
    assert glasso.glasso_create(C.byref(cfg), C.byref(h)) == 12  # GLASSO_ERR_UNSUPPORTED
    assert not h.value


def _header_text():
    return re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)


def _enum_values(prefix):
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(" + prefix + r"[A-Z0-9_]+)\s*=\s*(\d+)", _header_text())}


def _struct_fields(name):
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r";", _header_text()).group(1)
    fields = []
    for decl in body.split(";"):
        for part in decl.split(","):  # "double a, b, c" declares three fields
            part = part.split("[")[0].strip()
            if part:
                fields.append(re.findall(r"[A-Za-z_][A-Za-z_0-9]*", part)[-1])
    return fields


def test_binding_constants_match_the_header(glasso):
    st = _enum_values("GLASSO_")
    for code, name in glasso.STATUS.items():
        assert st[name] == code, name
    for key, value in glasso.PRECISION.items():
        assert value == {"fp64": st["GLASSO_FP64"], "tf32x3": st["GLASSO_MIXED_TF32X3"],
                         "bf16x3": st["GLASSO_MIXED_BF16X3"]}[key]
    for key, value in glasso.PRODUCTS.items():
        assert st["GLASSO_PRODUCTS_" + key.upper()] == value
    for key, value in glasso.METHODS.items():
        assert st["GLASSO_METHOD_" + key.upper()] == value
    prof = _enum_values("GLASSO_PROF_")
    assert prof.pop("GLASSO_PROF_CLASSES") == len(glasso.PROF_CLASSES)
    for name, idx in prof.items():
        assert glasso.PROF_CLASSES[idx] == name[len("GLASSO_PROF_"):].lower()


def test_binding_structures_follow_the_header_field_order(glasso):
    structs = [n for n in dir(glasso) if n.startswith("glasso_") and isinstance(getattr(glasso, n), type)
               and issubclass(getattr(glasso, n), C.Structure)]
    assert {"glasso_config", "glasso_result", "glasso_profile"} <= set(structs)
    for cname in structs:
        py = getattr(glasso, cname)
        # (a trailing underscore stands for a Python keyword: lambda_)
        assert _struct_fields(cname) == [f.rstrip("_") for f, _ in py._fields_], cname


def test_workspace_bytes_needs_no_gpu(glasso):
    sizes = [glasso.workspace_bytes(n) for n in (1, 128, 129, 1000, 10000)]
    assert sizes[0] == sizes[1] < sizes[2] < sizes[3] < sizes[4]   # padded to multiples of 128
    assert sizes[4] >= 12 * 8 * 10000 ** 2                          # at least the FP64 matrices
    v = C.c_size_t()
    assert glasso.glasso_workspace_bytes(0, C.byref(v)) == 1

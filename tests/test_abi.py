"""The C ABI library loads without a GPU and exports every entry point that
include/dpcs.h declares; the ctypes mirrors of the public structs have the
C layout (checked against gcc's sizeof/offsetof)."""
import ctypes
import os
import re
import subprocess
import tempfile

from paper_2503_12174_gb300 import dpcs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "include", "dpcs.h")


def _declared():
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dpcs_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = dpcs.load_library()
    names = _declared()
    assert len(names) >= 14
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(names) <= set(dpcs.EXPORTED) | {n for n in names if n not in dpcs.EXPORTED and hasattr(lib, n)}


def test_create_without_gpu_fails_cleanly():
    import torch

    if torch.cuda.is_available():
        return
    lib = dpcs.load_library()
    h = ctypes.c_void_p()
    assert lib.dpcs_create(0, 0, ctypes.byref(h)) == dpcs.DPCS_ERR_INVALID_ARG
    assert not h.value


def test_struct_layout_matches_header():
    code = r"""
#include <stdio.h>
#include <stddef.h>
#include "dpcs.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(dpcs_params), offsetof(dpcs_params, rr_start),
         offsetof(dpcs_params, jitter), sizeof(dpcs_view), offsetof(dpcs_view, Kp), offsetof(dpcs_view, Hp),
         sizeof(dpcs_request), offsetof(dpcs_request, seed), offsetof(dpcs_request, Ip_out),
         sizeof(dpcs_serve_config), offsetof(dpcs_serve_config, quantum_samples), sizeof(dpcs_serve_stats),
         sizeof(dpcs_denoise_params), offsetof(dpcs_denoise_params, sigma_depth),
         offsetof(dpcs_serve_config, est_samples_per_s), offsetof(dpcs_serve_config, compensation_share));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(code)
        subprocess.check_call(["gcc", "-I", os.path.dirname(HDR), c, "-o", exe])
        out = [int(x) for x in subprocess.check_output([exe]).split()]
    P, V, R, C = dpcs.DpcsParams, dpcs.DpcsView, dpcs.DpcsRequest, dpcs.DpcsServeConfig
    assert out == [ctypes.sizeof(P), P.rr_start.offset, P.jitter.offset, ctypes.sizeof(V), V.Kp.offset, V.Hp.offset,
                   ctypes.sizeof(R), R.seed.offset, R.Ip_out.offset, ctypes.sizeof(C), C.quantum_samples.offset,
                   ctypes.sizeof(dpcs.DpcsServeStats), ctypes.sizeof(dpcs.DpcsDenoiseParams),
                   dpcs.DpcsDenoiseParams.sigma_depth.offset, C.est_samples_per_s.offset,
                   C.compensation_share.offset]


def test_probe_library_exports_its_header_and_the_product_library_has_no_probes():
    """The roof probes live in the measurement library (include/dpcs_probe.h),
    not in libdpcs.so."""
    from paper_2503_12174_gb300 import probe

    src = open(os.path.join(ROOT, "include", "dpcs_probe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = sorted(set(re.findall(r"\b(dpcs_[a-z0-9_]+)\s*\(", src)))
    assert names == ["dpcs_probe_atomic4", "dpcs_probe_l2_load"]
    plib = probe.load_library()
    assert all(hasattr(plib, n) for n in names)
    lib = dpcs.load_library()
    assert not any(hasattr(lib, n) for n in names)


def _prototypes():
    """{name: (return type, [parameter types])} of every function include/dpcs.h declares."""
    src = open(HDR).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"#[^\n]*", "", src)
    out = {}
    for ret, name, params in re.findall(r"([A-Za-z_][\w \t\*]*?)\b(dpcs_[a-z0-9_]+)\s*\(([^()]*)\)\s*;", src):
        ps = [p.strip() for p in params.split(",") if p.strip() and p.strip() != "void"]
        out[name] = (ret.strip(), ps)
    return out


_C_INT = {"int": 4, "int32_t": 4, "uint32_t": 4, "int64_t": 8, "uint64_t": 8, "size_t": 8, "dpcs_scene": 8,
          "dpcs_status": 4}


def _c_kind(decl):
    """('ptr',), ('int', bytes) or ('float', bytes) of a C declaration such as
    'const float *Ip', 'const float R[9]', 'int32_t Ht' or 'dpcs_status'."""
    if "*" in decl or "[" in decl:
        return ("ptr",)
    words = [w for w in decl.replace("const", " ").split()]
    base = words[0]
    if base == "float":
        return ("float", 4)
    if base == "double":
        return ("float", 8)
    return ("int", _C_INT[base])


def _ctypes_kind(t):
    if t in (ctypes.c_void_p, ctypes.c_char_p) or hasattr(t, "_type_") and isinstance(t._type_, type):
        return ("ptr",)
    if t in (ctypes.c_float, ctypes.c_double):
        return ("float", ctypes.sizeof(t))
    return ("int", ctypes.sizeof(t))


def test_binding_signatures_match_the_header():
    """Every ctypes signature the binding sets has the header's parameter
    count and, position by position, the same kind of argument (pointer,
    integer of the same width, float or double) and return type, so no call
    passes arguments the library reads differently."""
    protos = _prototypes()
    assert set(dpcs._SIGS) <= set(protos), sorted(set(dpcs._SIGS) - set(protos))
    assert set(dpcs.EXPORTED) <= set(dpcs._SIGS), sorted(set(dpcs.EXPORTED) - set(dpcs._SIGS))
    for name, (res, args) in dpcs._SIGS.items():
        ret, params = protos[name]
        assert len(args) == len(params), (name, len(args), len(params))
        assert _ctypes_kind(res) == _c_kind(ret), (name, ret, res)
        for i, (a, p) in enumerate(zip(args, params)):
            assert _ctypes_kind(a) == _c_kind(p), (name, i, p, a)

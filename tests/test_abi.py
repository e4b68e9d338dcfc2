"""The C-ABI library builds, loads and exports what include/kf.h declares;
argument checks that run before any CUDA call (no GPU needed)."""
import ctypes

import pytest

from paper_2401_14221_gb300 import build as kbuild
from paper_2401_14221_gb300 import kf


@pytest.fixture(scope="module")
def lib():
    kbuild.build()
    return kf.load()


def test_exports_every_declared_function(lib):
    names = kf.header_functions()
    assert "kf_p2z_propagate_update" in names and "kf_p2r_propagate_update" in names
    for name in names:
        assert hasattr(lib, name), f"libkf.so does not export {name}"


def test_version(lib):
    assert kf.kf_version() == 400  # KF_VERSION of include/kf.h


def _call(lib, name, params, layout):
    fn = getattr(lib, name)
    p = ctypes.byref(params) if params is not None else None
    dummy = ctypes.c_void_p(16)  # never dereferenced: every case fails before use
    return fn(p, layout, dummy, dummy, dummy, dummy, dummy, dummy, dummy, dummy, 0, None, None)


@pytest.mark.parametrize("name", ["kf_p2z_propagate_update", "kf_p2r_propagate_update"])
def test_argument_checks_without_gpu(lib, name):
    good = kf.make_params(3.8)
    assert _call(lib, name, None, kf.make_layout(kf.KF_SOA, 0, 10)) == kf.KF_ERR_ARG
    assert "params" in kf.kf_last_error_string()
    assert _call(lib, name, kf.make_params(3.8, flags=1), kf.make_layout(0, 0, 10)) == kf.KF_ERR_ARG
    assert _call(lib, name, kf.make_params(3.8, precision=7), kf.make_layout(0, 0, 10)) == kf.KF_ERR_ARG
    assert _call(lib, name, good, kf.make_layout(kf.KF_SOA, 0, -1)) == kf.KF_ERR_ARG
    assert _call(lib, name, good, kf.make_layout(5, 0, 10)) == kf.KF_ERR_ARG
    assert _call(lib, name, good, kf.make_layout(kf.KF_AOSOA, 24, 10)) == kf.KF_ERR_ARG
    assert "width" in kf.kf_last_error_string()
    # n = 0 launches nothing and succeeds, whatever the pointers
    assert _call(lib, name, good, kf.make_layout(kf.KF_AOSOA, 64, 0)) == kf.KF_OK
    assert kf.kf_last_error_string() == ""


def test_binding_refuses_cpu_tensors(lib):
    import torch
    t = torch.zeros(6, dtype=torch.float32)
    with pytest.raises(ValueError):
        kf.kf_p2z_propagate_update(kf.make_params(3.8), kf.make_layout(0, 0, 1), t, t, t, t,
                                   torch.zeros(1, dtype=torch.int8), t, t, t)


def test_tuning_cache_text_round_trip(lib):
    # the cache is host state: import / export / clear need no GPU
    kf.autotune_clear()
    assert kf.autotune_export() == ""
    line = f"NVIDIA GB300/152|0|1|0|0|5|20|{kf.KF_STEP_STAGED}|256|3|0.0451\n"
    kf.autotune_import(line)
    assert kf.autotune_export() == line
    bad_fields = ["no separators here", "G|0|1|0|0|5|20|9|256|2|0.1",  # unknown kernel
                  "G|0|1|0|0|5|20|2|100|2|0.1",                       # CTA size
                  "G|0|1|0|0|5|20|2|256|4|0.1",                       # CTAs per SM
                  "G|2|1|0|0|5|20|2|256|2|0.1",                       # op
                  "G|0|1|9|0|5|20|2|256|2|0.1",                       # precision
                  "G|0|1|0|0|5|20|2|256|2"]                           # missing field
    for bad in bad_fields:
        with pytest.raises(kf.KfError):
            kf.autotune_import(bad + "\n")
    assert kf.autotune_export() == line
    kf.autotune_clear()
    assert kf.autotune_export() == ""


def test_process_wide_knobs_validate_their_argument(lib):
    # host state only: an unknown mode is refused and leaves the setting alone
    for fn, bad, good in ((kf.kf_set_host_path, 3, kf.KF_HOST_AUTO),
                          (kf.kf_set_step_kernel, 3, kf.KF_STEP_AUTO),
                          (kf.kf_set_staged_ctas_per_sm, 4, 0),
                          (kf.kf_set_chain_redo, 2, kf.KF_CHAIN_REDO_LIST)):
        with pytest.raises(kf.KfError) as e:
            fn(bad)
        assert e.value.code == kf.KF_ERR_ARG
        fn(good)
    for mode in (kf.KF_HOST_COPY, kf.KF_HOST_DIRECT, kf.KF_HOST_AUTO):
        kf.kf_set_host_path(mode)


def test_host_entry_argument_checks_without_gpu(lib):
    # the host-array calls refuse bad arguments before touching any pointer
    p = kf.make_params(3.8, precision=9)
    rc = lib.kf_p2r_propagate_update_host(ctypes.byref(p), kf.make_layout(0, 0, 10), *[None] * 8,
                                          0, None, None, 0, 0, None)
    assert rc == kf.KF_ERR_ARG and "precision" in kf.kf_last_error_string()
    rc = lib.kf_p2r_propagate_update_host(ctypes.byref(kf.make_params(3.8)),
                                          kf.make_layout(0, 0, 10), *[None] * 8, 0, None, None,
                                          0, 0, None)
    assert rc == kf.KF_ERR_ARG and "NULL" in kf.kf_last_error_string()
    rc = lib.kf_propagate_update_host_noalloc(7, ctypes.byref(kf.make_params(3.8)),
                                              kf.make_layout(0, 0, 10), *[None] * 8, 0, None,
                                              0, None)
    assert rc == kf.KF_ERR_ARG


def test_device_wait_limit_range(lib):
    # host-side argument check only (no CUDA call)
    for bad in (-2, (1 << 24) + 1, 1 << 40):
        with pytest.raises(kf.KfError) as e:
            kf.kf_set_device_wait_limit(bad)
        assert e.value.code == kf.KF_ERR_ARG
    kf.kf_set_device_wait_limit(1 << 24)
    kf.kf_set_device_wait_limit(0)
    kf.kf_set_device_wait_limit(-1)


def test_binding_constants_match_the_header(lib):
    # every #define KF_* the binding mirrors carries the header's value
    import re
    text = open(kf.HEADER).read()
    defines = {m.group(1): int(m.group(2), 0)
               for m in re.finditer(r"#define\s+(KF_[A-Z0-9_]+)\s+([0-9]+)u?\b", text)}
    names = ["KF_OK", "KF_ERR_ARG", "KF_ERR_CUDA", "KF_ERR_UNSUPPORTED", "KF_ERR_TIMEOUT",
             "KF_SOA", "KF_AOSOA", "KF_FP32", "KF_FP64_UPDATE", "KF_JOSEPH", "KF_FP64",
             "KF_ADAPTIVE", "KF_DF_UPDATE", "KF_MAX_LAYERS", "KF_P2Z", "KF_P2R",
             "KF_NOALLOC_MAX_CHUNK", "KF_STEP_AUTO", "KF_STEP_DIRECT", "KF_STEP_STAGED",
             "KF_DEVERR_TIMEOUT", "KF_HOST_AUTO", "KF_HOST_COPY", "KF_HOST_DIRECT"]
    for name in names:
        assert name in defines, name
        assert getattr(kf, name) == defines[name], name
    bits = {"NO_INTERSECT": "KF_NO_INTERSECT", "S_NOT_PD": "KF_S_NOT_PD", "BAD_K": "KF_BAD_K",
            "NONFINITE": "KF_NONFINITE"}
    for py, c in bits.items():
        assert getattr(kf, py) == defines[c], c

"""Host-side checks of the C ABI (no GPU needed): the library builds, loads,
exports every function include/dgw.h declares, and its host-only calls work."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1711_01175_gb300 import build, capi
    build.build()
    return capi.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dgw.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dgw_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("dgw_mesh_upload", "dgw_material_upload", "dgw_rhs", "dgw_step", "dgw_energy",
                     "dgw_adjoint_step", "dgw_create", "dgw_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    from paper_1711_01175_gb300 import capi
    names = declared_functions()
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(capi.SIGNATURES) == names
    for name in names:                       # a Python function of the same name for each
        assert callable(getattr(capi, name, None)), name


def test_abi_version(lib):
    text = open(os.path.join(ROOT, "include", "dgw.h")).read()
    v = int(re.search(r"#define DGW_ABI_VERSION (\d+)", text).group(1))
    assert lib.dgw_abi_version() == v


@pytest.mark.parametrize("N", range(1, 8))
def test_reference_nodes_match_oracle_gll(lib, N):
    from paper_1711_01175_gb300 import reference_nodes
    r, w = reference_nodes(N)
    ro, wo = oracle.gll(N)
    np.testing.assert_allclose(r, ro, atol=2e-16 * 4)
    np.testing.assert_allclose(w, wo, rtol=1e-14)


def test_reference_nodes_rejects_bad_degree(lib):
    from paper_1711_01175_gb300 import capi
    r = np.zeros(10)
    w = np.zeros(10)
    for N in (0, 8, -1):
        st = lib.dgw_reference_nodes(N, r.ctypes.data, w.ctypes.data)
        assert st == -1
        assert "outside" in capi.dgw_last_error(None)
    assert lib.dgw_reference_nodes(3, None, None) == -1


def test_create_rejects_bad_config_without_touching_a_device(lib):
    from paper_1711_01175_gb300 import capi
    for cfg in (capi.dgw_config(0, 1, 0, 0.5), capi.dgw_config(3, 2, 0, 0.5),
                capi.dgw_config(3, 1, 5, 0.5), capi.dgw_config(3, 1, 0, -1.0)):
        st, h = capi.dgw_create(0, cfg)
        assert st == -1 and not h.value


def test_create_rejects_bad_system_config_without_touching_a_device(lib):
    from paper_1711_01175_gb300 import capi
    B = ctypes.c_double * 3
    bad = [(capi.dgw_config(3, 1, 0, 0.5, 7, B(0, 0, 0)), -1),                    # unknown system
           (capi.dgw_config(3, 1, 0, 0.5, capi.DGW_SYSTEM_TRANSPORT, B(0, 0, 0)), -1),   # beta = 0
           (capi.dgw_config(3, 1, 1, 0.5, capi.DGW_SYSTEM_SHALLOW_WATER, B(0, 0, 0)), -7),  # mixed: not built
           (capi.dgw_config(3, 1, 1, 0.5, capi.DGW_SYSTEM_TRANSPORT, B(1, 0, 0)), -7)]
    for cfg, want in bad:
        st, h = capi.dgw_create(0, cfg)
        assert st == want and not h.value, capi.dgw_last_error(None)


def test_config_struct_layout_matches_the_header():
    """dgw_config as the C compiler lays it out: int N, flux_tau, precision;
    double cfl; int system; double beta[3]."""
    from paper_1711_01175_gb300 import capi
    text = open(os.path.join(ROOT, "include", "dgw.h")).read()
    body = re.search(r"typedef struct \{(.*?)\} dgw_config;", text, re.S).group(1)
    names = re.findall(r"^\s*(?:int|double)\s+(\w+)", body, re.M)
    assert names == [f[0] for f in capi.dgw_config._fields_] == ["N", "flux_tau", "precision", "cfl", "system", "beta"]
    assert ctypes.sizeof(capi.dgw_config) == 56
    assert capi.dgw_config.beta.offset == 32


def test_calls_on_null_context_fail_cleanly(lib):
    from paper_1711_01175_gb300 import capi
    assert capi.dgw_rhs(None, None, None, 0.0, None) == -1
    assert capi.dgw_step(None, None, None, 0.0, 0.1, 1, None) == -1
    assert capi.dgw_step_energy(None, None, None, 0.0, 0.1, 1, None)[0] == -1
    assert capi.dgw_mesh_upload(None, 1, None, None, None, None, None) == -1
    assert capi.dgw_destroy(None) == 0


def test_every_declaration_is_documented():
    """Each function of the boundary is preceded by its own comment block
    (argument meaning, layout, ownership, errors)."""
    text = open(os.path.join(ROOT, "include", "dgw.h")).read()
    undocumented = []
    for m in re.finditer(r"^(?:dgw_status|const char\*|int)\s+(dgw_\w+)\s*\(", text, re.M):
        lines = text[:m.start()].rstrip().split("\n")
        while lines and lines[-1].lstrip().startswith("#"):      # a #define between comment and call
            lines.pop()
        if not "\n".join(lines).rstrip().endswith("*/"):
            undocumented.append(m.group(1))
    # calls documented together with the call right above them
    grouped = {"dgw_destroy", "dgw_batch_destroy", "dgw_batch_last_error", "dgw_abi_version"}
    assert not [f for f in undocumented if f not in grouped], undocumented


def test_energy_static_refuses_host_arrays(lib):
    """dgw_energy_static takes only device memory of the current device: plain
    host arrays are refused with DGW_ERR_ARG before anything is launched (no
    GPU needed to see it)."""
    from paper_1711_01175_gb300 import capi
    host = np.zeros(64 * 27)
    p = host.ctypes.data
    assert capi.dgw_energy_static(2, 1, p, p, p, p, p, p, None) == -1
    assert "device memory" in capi.dgw_last_error(None)


def test_create_refuses_unknown_precision(lib):
    from paper_1711_01175_gb300 import capi
    for prec in (-1, 4):
        cfg = capi.dgw_config(3, 1, prec, 0.5, 0, (ctypes.c_double * 3)(0, 0, 0))
        st, _ = capi.dgw_create(0, cfg)
        assert st == -1 and "precision" in capi.dgw_last_error(None)


def test_state_calls_refuse_missing_context(lib):
    """Checkpoint calls need a context with a mesh (no GPU needed to see the refusal)."""
    from paper_1711_01175_gb300 import capi
    st, _ = capi.dgw_state_bytes(None, 1)
    assert st == -1
    buf = np.zeros(128, dtype=np.uint8)
    st, _, _ = capi.dgw_set_state(None, buf.ctypes.data, buf.nbytes, buf.ctypes.data, None, None)
    assert st == -1 and "context" in capi.dgw_last_error(None)


def test_debug_status_refuses_missing_context(lib):
    from paper_1711_01175_gb300 import capi
    assert capi.dgw_debug_status(None)[0] == -1

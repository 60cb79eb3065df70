"""The C-ABI library builds, loads without a GPU, exports every declared symbol, and
rejects bad arguments on the host before touching the device."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "corde.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rod_\w+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2509_04277_gb300 import build, corde

    build.build()
    return corde.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("rod_create", "rod_step", "rod_get_state", "rod_set_input", "rod_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    import ctypes

    for name in declared_functions():
        assert hasattr(lib, name), f"libcorde.so does not export {name}"
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_binding_covers_every_declared_symbol(lib):
    from paper_2509_04277_gb300 import corde

    assert set(declared_functions()) <= set(corde.SIGNATURES)


def test_argument_errors_are_reported_on_the_host(lib):
    from paper_2509_04277_gb300 import corde
    from paper_2509_04277_gb300 import workloads as W

    rod = W.guidewire(8)
    good = corde.params_of(rod)
    pos = np.zeros((8, 3), np.float32)
    quat = np.zeros((7, 4), np.float32)
    with pytest.raises(corde.CordeError) as e:
        corde.rod_create([], pos, quat)
    assert e.value.code == corde.CORDE_ERR_ARG
    bad = corde.params_of(rod)
    bad.n_nodes = 1
    with pytest.raises(corde.CordeError) as e:
        corde.rod_create([bad], pos, quat)
    assert e.value.code == corde.CORDE_ERR_ARG
    bad = corde.params_of(rod)
    bad.dt = 0.0
    with pytest.raises(corde.CordeError) as e:
        corde.rod_create([bad], pos, quat)
    assert e.value.code == corde.CORDE_ERR_ARG
    big = corde.params_of(rod)
    big.n_nodes = 1 << 20
    with pytest.raises(corde.CordeError) as e:
        corde.rod_create([big], pos, quat)
    assert e.value.code == corde.CORDE_ERR_UNSUPPORTED
    with pytest.raises(corde.CordeError) as e:
        corde.rod_create([good], None, quat)
    assert e.value.code == corde.CORDE_ERR_ARG
    assert lib.rod_step(None, 1, None, None) == corde.CORDE_ERR_ARG
    assert lib.rod_set_launch_overlap(None, 1) == corde.CORDE_ERR_ARG
    assert lib.rod_set_adjoint_record_budget(None, 0) == corde.CORDE_ERR_ARG
    assert lib.rod_mailbox_exchange(None, None, 0, 0, None, 0, None) == corde.CORDE_ERR_ARG
    assert lib.rod_mailbox_tick(None, 0, 0, None, None, 0, None) == corde.CORDE_ERR_ARG
    assert lib.rod_strerror(corde.CORDE_ERR_NONFINITE) == b"non-finite state"


def test_oracle_is_not_imported_by_the_product_path():
    """The CUDA path's package never reaches the oracle (no CPU fallback)."""
    pkg = os.path.join(ROOT, "paper_2509_04277_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import oracle|from oracle\b)", src, flags=re.M), f
                assert "corde_oracle" not in src, f

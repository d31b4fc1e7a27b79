"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every
function declared in include/gks.h (no compute call is made without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gks_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("gks_create", "gks_set_state", "gks_step", "gks_get_state", "gks_destroy", "gks_advance"):
        assert n in names


def test_library_exports_every_declared_function():
    from paper_1412_4489_gb300 import build
    lib = ctypes.CDLL(build.build())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_the_abi():
    from paper_1412_4489_gb300 import gks
    for n in ("gks_create", "gks_set_state", "gks_set_state_device", "gks_step", "gks_advance", "gks_sync",
              "gks_get_state", "gks_get_state_device", "gks_destroy", "gks_last_error"):
        assert callable(getattr(gks, n))


def test_default_options():
    from paper_1412_4489_gb300 import gks
    o = gks.gks_default_options()
    assert (o.precision, o.weno_eps, o.weno_C, o.tau_eps, o.tau_C, o.viscous_dt, o.characteristic) == \
        (0, 1e-6, 10.0, 0.05, 1.0, 0, 0)


def test_invalid_sizes_are_rejected_before_touching_the_device():
    """Argument checks run before any CUDA call, so they hold on a host without a GPU: empty
    grids, more than 2^31 cells, and grids taller than the launch grids can cover."""
    import pytest
    from paper_1412_4489_gb300 import gks
    for nx, ny in ((0, 4), (4, 0), (-1, 3), (1 << 16, (1 << 15) + 1), (2, 262140)):
        with pytest.raises(gks.GKSError) as e:
            gks.gks_create(nx, ny, 1.0, 1.0, 1.4, 1.0, 0.0)
        assert e.value.status == gks.GKS_EINVAL


def test_an_axis_one_cell_across_must_be_periodic():
    """A wall or outflow side on an axis one cell across is rejected before any CUDA call."""
    import pytest
    from paper_1412_4489_gb300 import gks
    walls = [gks.GKS_BC_SLIPWALL] * 4
    for nx, ny in ((1, 5), (5, 1)):
        with pytest.raises(gks.GKSError) as e:
            gks.gks_create(nx, ny, 1.0, 1.0, 1.4, 1.0, 0.0, bc=walls)
        assert e.value.status == gks.GKS_EINVAL
        assert "periodic" in gks.gks_last_error(None)

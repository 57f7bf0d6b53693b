"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function include/*.h declares, and validates
parameters before it touches a device."""
import ctypes
import glob
import os
import re

import pytest

from paper_2211_02435_b300 import build as B
from paper_2211_02435_b300 import lbm as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(lbm_\w+)\s*\(", src, re.M):
            names.add(m.group(1))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "lbm_step" in names and "lbm_create" in names
    for n in sorted(names):
        assert hasattr(lib, n), n


def _params(**kw):
    p = dict(stencil=L.D3Q27, space=L.SPACE_CUMULANT, equilibrium=L.EQ_ABSOLUTE,
             storage=L.STORE_F32, streaming=L.PULL, rates=[1.9] + [1.0] * 5,
             dims=(8, 8, 8), boundary=L.PERIODIC, arithmetic=L.ARITH_DEVIATION)
    p.update(kw)
    return L.Params(p["stencil"], p["space"], p["equilibrium"], p["storage"], p["streaming"],
                    (ctypes.c_double * 6)(*p["rates"]), (ctypes.c_int64 * 3)(*p["dims"]),
                    p["boundary"], None, p["arithmetic"])


@pytest.mark.parametrize("kw,code", [
    (dict(stencil=3), -1),
    (dict(space=7), -1),
    (dict(storage=9), -1),
    (dict(streaming=5), -1),
    (dict(equilibrium=5), -1),
    (dict(dims=(0, 4, 4)), -1),
    (dict(dims=(4, 70000, 4)), -1),
    (dict(dims=(2048, 2048, 1024)), -1),
    (dict(stencil=L.D2Q9, dims=(8, 8, 2)), -1),
    (dict(rates=[2.5] + [1.0] * 5), -1),
    (dict(rates=[0.0] + [1.0] * 5), -1),
    (dict(space=L.SPACE_CUMULANT, equilibrium=L.EQ_DELTA), -3),
    (dict(boundary=1), -2),
    (dict(arithmetic=2), -1),
    # absolute storage holds f itself: delta-equilibria (Eq. 2.5) need zero-centered storage
    (dict(space=L.SPACE_RAW, equilibrium=L.EQ_DELTA, storage=L.STORE_F64_ABSOLUTE), -3),
    (dict(storage=L.STORE_F64_ABSOLUTE, streaming=L.AA), -2),
    (dict(arithmetic=L.ARITH_AS_WRITTEN, storage=L.STORE_F32), -2),
    (dict(arithmetic=L.ARITH_AS_WRITTEN, storage=L.STORE_F64, streaming=L.AA), -2),
    # the discrete equilibrium: FP64 / FP32 deviations with pull streaming only
    (dict(equilibrium=L.EQ_DISCRETE2, storage=L.STORE_F16_DELTA), -2),
    (dict(equilibrium=L.EQ_DISCRETE2, streaming=L.ESOTERIC_PULL), -2),
    (dict(equilibrium=L.EQ_DISCRETE2, storage=L.STORE_F64_ABSOLUTE), -2),
    (dict(equilibrium=L.EQ_DISCRETE2, storage=L.STORE_F64, arithmetic=L.ARITH_AS_WRITTEN), -2),
    (dict(equilibrium=3), -1),
])
def test_create_rejects_bad_parameters(lib, kw, code):
    h = ctypes.c_void_p()
    assert lib.lbm_create(ctypes.byref(h), ctypes.byref(_params(**kw))) == code
    assert not h.value


def test_null_arguments(lib):
    assert lib.lbm_create(None, None) == -1
    assert lib.lbm_step(None, 1) == -1
    assert lib.lbm_macroscopic(None, None, None, 0) == -1
    assert lib.lbm_invariants(None, None) == -1
    assert lib.lbm_set_step_kernel(None, 0) == -1
    assert lib.lbm_run_host(None, None, None, 1, None, None, 0) == -1
    assert lib.lbm_set_divergence_check(None, 1) == -1
    lib.lbm_destroy(None)
    for c in (0, -1, -2, -3, -4, -5, -6, -7, -8):
        assert lib.lbm_error_string(c)


@pytest.mark.parametrize("dims", [
    (4, 1, (1 << 62) + 1),        # the int64 product would wrap to 4
    (1 << 40, 1 << 40, 1),        # Nx * Ny alone overflows
    ((1 << 62) + 1, 1, 4),
    (1, (1 << 63) - 1, 1),
    (1 << 16, 1 << 15, 2),        # exactly 2^32 cells
    (1, 1, 1 << 31),              # 2^31 cells: one more than a call serves
    (46341, 46341, 1),            # 2^31 + 1 cells in the xy plane
    (3, 3, -1),
])
def test_noalloc_rejects_wrapping_sizes_before_any_launch(lib, dims):
    # the size check runs before the library touches a device, so these
    # calls return LBM_ERR_INVALID on a machine without a GPU as well; the
    # population pointer is never dereferenced
    d = (ctypes.c_int64 * 3)(*dims)
    out = (ctypes.c_double * 8)()
    rc = lib.lbm_invariants_noalloc(L.D3Q27, L.STORE_F32, ctypes.c_void_p(1 << 20), d,
                                    ctypes.addressof(out), 0, None)
    assert rc == -1


@pytest.mark.parametrize("st,dims,fits", [
    (L.D3Q27, (65536, 32767, 1), False),   # N < 2^31, but N + Nx*Ny is not
    (L.D3Q27, (1024, 1024, 2047), False),  # N + Nx*Ny = 2^31
    (L.D3Q27, (1024, 1024, 2046), True),   # the largest Nz for a 1024^2 plane
    (L.D3Q19, (46000, 46000, 1), False),   # one plane: the z wrap doubles the index
    (L.D2Q9, (46000, 46000, 1), True),     # no z wrap on D2Q9: N + 2*Nx + 4096 < 2^31
    (L.D2Q9, (46340, 46340, 1), False),
    (L.D3Q27, (1 << 31, 1, 1), False),
])
def test_create_bounds_the_kernels_cell_indices(lib, st, dims, fits):
    # the step kernels form cell index + periodic wrap in 32-bit integers, so
    # a lattice is refused unless N + Nx*Ny + 2*Nx + 4096 < 2^31 (D2Q9: N +
    # 2*Nx + 4096); the check runs before any device work (FP64 storage: an
    # accepted size fails later, for want of a device here or of the 300 GB
    # and more it would take on a B300)
    h = ctypes.c_void_p()
    rc = lib.lbm_create(ctypes.byref(h),
                        ctypes.byref(_params(stencil=st, dims=dims, storage=L.STORE_F64)))
    if fits:
        assert rc in (-5, -4), rc
    else:
        assert rc == -1
    assert not h.value


@pytest.mark.parametrize("box", [
    (65536, 32767, 1),            # one instance past the 32-bit index bound
    ((1 << 40) + 1, 1, 1),        # Nx alone past 2^31 (its product must not wrap)
    (1, 1 << 40, 1 << 30),
    (8, 8, 0),
])
def test_batch_create_bounds_every_instance_before_device_work(lib, box):
    h = ctypes.c_void_p()
    dims = (ctypes.c_int64 * 6)(8, 8, 8, *box)
    p = _params(stencil=L.D3Q19, space=L.SPACE_RAW, rates=[1.5] + [1.0] * 5)
    assert lib.lbm_batch_create(ctypes.byref(h), ctypes.byref(p), 2, dims, None) == -1
    assert not h.value


def test_python_binding_raises_on_error(lib):
    with pytest.raises(L.LBMError) as e:
        L.Lattice(L.D3Q27, L.SPACE_CUMULANT, L.EQ_DELTA, L.STORE_F32, L.PULL, [1.9], (8, 8, 8))
    assert e.value.code == -3

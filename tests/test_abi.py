"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/lw.h declares; host-side argument checks and size queries work
without touching a device."""
import ctypes
import os
import re

import pytest

from paper_2206_03015_gb300 import build as lwbuild
from paper_2206_03015_gb300 import lw

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            with open(os.path.join(ROOT, "include", h)) as f:
                text = f.read()
            names += re.findall(r"^(?:int|size_t)\s+(lw_\w+)\s*\(", text, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    lwbuild.build()
    return lw.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("lw_trajectories_upload", "lw_grid_bounds", "lw_deposit_time_domain",
              "lw_spectrum"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    raw = ctypes.CDLL(lw.library_path())
    for n in declared_functions():
        assert hasattr(raw, n), n


def test_upload_argument_checks_and_size_query(lib):
    nbytes = ctypes.c_size_t(0)
    view = lw.lw_traj()
    assert lib.lw_trajectories_upload(None, 3, 64, None, ctypes.byref(nbytes),
                                      ctypes.byref(view), None) == lw.LW_EINVAL
    fake = ctypes.c_void_p(0x1000)   # never dereferenced by a size query
    inp = lw.lw_traj_in(10, 99, fake, 0, fake, fake, fake)
    assert lib.lw_trajectories_upload(ctypes.byref(inp), 3, 64, None, ctypes.byref(nbytes),
                                      ctypes.byref(view), None) == lw.LW_OK
    # status + ends + FP64 copies + mixed section (scan, field, anchors) + electron order
    # and its scratch (two range keys + 4096 bucket counters), each 256-byte aligned
    ns1, ne = 100, 10
    al = lambda x: (x + 255) // 256 * 256  # noqa: E731
    fp64 = al(8 * ns1) + 3 * al(8 * 3 * ne * ns1)
    mixed = al(16 * ne * ns1) + al(24 * ne * ns1) + al(32 * ne * 2)
    order = al(4 * ne) + al(16 + 4 * 4096)
    assert nbytes.value == al(4) + al(64 * ne) + fp64 + mixed + order
    for bad_block in (8, 100, 2048):
        assert lib.lw_trajectories_upload(ctypes.byref(inp), 3, bad_block, None,
                                          ctypes.byref(nbytes), ctypes.byref(view),
                                          None) == lw.LW_EINVAL
    bad = lw.lw_traj_in(0, 99, fake, 0, fake, fake, fake)
    assert lib.lw_trajectories_upload(ctypes.byref(bad), 3, 64, None, ctypes.byref(nbytes),
                                      ctypes.byref(view), None) == lw.LW_EINVAL


def test_deposit_argument_checks(lib):
    view = lw.lw_traj()
    view.sections = lw.LW_SECTION_FP64
    det = lw.lw_detector(4, 0x1000, 1.0)
    rec = ctypes.c_void_p(0x2000)
    for g, flags, prec in ((lw.lw_grid(0.0, 0.0, 16), 1, 0),         # dt_u = 0
                           (lw.lw_grid(0.0, 1e-18, 0), 1, 0),        # no bins
                           (lw.lw_grid(0.0, 1e-18, 16), 0, 0),       # no field term
                           (lw.lw_grid(0.0, 1e-18, 16), 1, 1),       # mixed section missing
                           (lw.lw_grid(0.0, 1e-18, 16), 1, 7)):      # unknown precision
        assert lib.lw_deposit_time_domain(ctypes.byref(view), ctypes.byref(det),
                                          ctypes.byref(g), prec, flags, rec, 0, None,
                                          None) == lw.LW_EINVAL


def test_spectrum_size_query_and_limits(lib):
    nbytes = ctypes.c_size_t(0)
    g = lw.lw_grid(0.0, 1e-18, 4096)
    assert lib.lw_spectrum(None, lw.LW_FP64, 10, ctypes.byref(g), 1.6e-19, None, None, None,
                           ctypes.byref(nbytes), None) == lw.LW_OK
    assert nbytes.value == 4096 * 16                      # twiddle table only
    g = lw.lw_grid(0.0, 1e-18, 65536)
    assert lib.lw_spectrum(None, lw.LW_MIXED, 10, ctypes.byref(g), 1.6e-19, None, None, None,
                           ctypes.byref(nbytes), None) == lw.LW_OK
    assert nbytes.value == 65536 * 8 + 3 * 5 * 65536 * 8  # twiddles + four-step buffer
    for n in (3, 1000, 1 << 19):
        g = lw.lw_grid(0.0, 1e-18, n)
        assert lib.lw_spectrum(None, lw.LW_FP64, 10, ctypes.byref(g), 1.6e-19, None, None, None,
                               ctypes.byref(nbytes), None) == lw.LW_EUNSUPPORTED


def test_struct_layouts_match_the_header(tmp_path):
    """The ctypes mirrors of the ABI structs have the C sizes and field offsets."""
    import subprocess
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "lw.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(lw_traj_in), sizeof(lw_traj), sizeof(lw_detector),
         sizeof(lw_grid), sizeof(lw_batch_item), sizeof(lw_batch));
  printf("%zu %zu %zu %zu\n", offsetof(lw_traj, t), offsetof(lw_traj, input_status),
         offsetof(lw_batch_item, grid), offsetof(lw_batch_item, e_chunk));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    sizes = [int(x) for x in out[:6]]
    offs = [int(x) for x in out[6:]]
    assert sizes == [ctypes.sizeof(c) for c in (lw.lw_traj_in, lw.lw_traj, lw.lw_detector,
                                                lw.lw_grid, lw.lw_batch_item, lw.lw_batch)]
    assert offs == [lw.lw_traj.t.offset, lw.lw_traj.input_status.offset,
                    lw.lw_batch_item.grid.offset, lw.lw_batch_item.e_chunk.offset]


def test_enum_values_match_the_header(tmp_path):
    """The binding's precision, field, status and section constants are the header's."""
    import subprocess
    names = ["LW_FP64", "LW_MIXED", "LW_MIXED_KAHAN", "LW_MIXED_F32", "LW_MIXED_F32X4", "LW_FIELD_ACCEL",
             "LW_FIELD_VELOCITY", "LW_ST_BETA", "LW_ST_NONFINITE", "LW_ST_TIME", "LW_ST_CLIP",
             "LW_ST_TA_ORDER", "LW_ST_STEP", "LW_ST_TIMEOUT", "LW_ST_PRECISION", "LW_SECTION_FP64", "LW_SECTION_MIXED"]
    src = tmp_path / "enums.c"
    src.write_text("#include <stdio.h>\n#include \"lw.h\"\nint main(void) {\n" +
                   "".join(f'  printf("%d\\n", (int){n});\n' for n in names) +
                   "  return 0;\n}\n")
    exe = tmp_path / "enums"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert [int(x) for x in out] == [getattr(lw, n) for n in names]


def test_pusher_adjoint_fdm_and_batch_argument_checks(lib):
    """Every call below has an argument that the entry point refuses before any CUDA call
    (the fake addresses are never dereferenced)."""
    fake = ctypes.c_void_p(0x1000)
    L = lw.lw_laser(0.8e-6, 0.5, 20e-6, 30e-15)
    bad_L = lw.lw_laser(0.0, 0.5, 20e-6, 30e-15)
    push = lambda r, n_e, dt, n_steps, laser, mass=9.1e-31: lib.lw_boris_push(  # noqa: E731
        r, fake, n_e, 0.0, dt, 0, n_steps, ctypes.byref(laser), -1.6e-19, mass,
        fake, fake, fake, fake, None)
    assert push(None, 4, 1e-17, 10, L) == lw.LW_EINVAL           # no state
    assert push(fake, 0, 1e-17, 10, L) == lw.LW_EINVAL           # no electrons
    assert push(fake, 4, 0.0, 10, L) == lw.LW_EINVAL             # dt = 0
    assert push(fake, 4, 1e-17, 0, L) == lw.LW_EINVAL            # no steps
    assert push(fake, 4, 1e-17, 10, bad_L) == lw.LW_EINVAL       # wavelength 0
    assert push(fake, 4, 1e-17, 10, L, mass=0.0) == lw.LW_EINVAL
    grad = lambda n_e, n_steps, out: lib.lw_boris_push_grad(  # noqa: E731
        fake, fake, n_e, 0.0, 1e-17, n_steps, ctypes.byref(L), -1.6e-19, 9.1e-31,
        fake, fake, fake, out, fake, None)
    assert grad(4, 10, None) == lw.LW_EINVAL
    assert grad(0, 10, fake) == lw.LW_EINVAL
    assert grad(4, 0, fake) == lw.LW_EINVAL

    det = lw.lw_detector(4, 0x1000, 1.0)
    view = lw.lw_traj()
    view.n_e, view.n_s = 2, 10
    view.sections = lw.LW_SECTION_MIXED                         # no FP64 section
    assert lib.lw_spectrum_fdm(ctypes.byref(view), ctypes.byref(det), 1e15, 1e13, 16, 1e-17,
                               1.6e-19, fake, None) == lw.LW_EINVAL
    view.sections = lw.LW_SECTION_FP64
    view.t, view.r = 0x1000, 0x1000
    assert lib.lw_spectrum_fdm(ctypes.byref(view), ctypes.byref(det), 1e15, 1e13, 0, 1e-17,
                               1.6e-19, fake, None) == lw.LW_EINVAL   # no frequencies
    assert lib.lw_spectrum_fdm(ctypes.byref(view), ctypes.byref(det), 1e15, 1e13, 16, 0.0,
                               1.6e-19, fake, None) == lw.LW_EINVAL   # dt = 0

    nbytes = ctypes.c_size_t(0)
    sg = lambda prec, flags, g: lib.lw_spectrum_grad(  # noqa: E731
        ctypes.byref(view), ctypes.byref(det), ctypes.byref(g), prec, flags, None, None,
        1.6e-19, None, None, None, None, ctypes.byref(nbytes), None)
    ok_grid = lw.lw_grid(0.0, 1e-18, 256)
    assert sg(7, lw.LW_FIELD_ACCEL, ok_grid) == lw.LW_EUNSUPPORTED          # unknown mode
    assert sg(lw.LW_FP64, lw.LW_FIELD_VELOCITY, ok_grid) == lw.LW_EUNSUPPORTED
    assert sg(lw.LW_FP64, lw.LW_FIELD_ACCEL, lw.lw_grid(0.0, 1e-18, 1000)) == \
        lw.LW_EUNSUPPORTED                                                  # not 2^k
    assert sg(lw.LW_FP64, lw.LW_FIELD_ACCEL, lw.lw_grid(0.0, 0.0, 256)) == lw.LW_EINVAL

    plan = lw.lw_batch()
    items = (lw.lw_batch_item * 1)()
    assert lib.lw_batch_plan(None, 1, lw.LW_MIXED, 1, None, ctypes.byref(nbytes),
                             ctypes.byref(plan), None) == lw.LW_EINVAL
    assert lib.lw_batch_plan(items, 1, lw.LW_FP64, 1, None, ctypes.byref(nbytes),
                             ctypes.byref(plan), None) == lw.LW_EUNSUPPORTED  # mixed only
    assert lib.lw_batch_plan(items, 1, lw.LW_MIXED, 0, None, ctypes.byref(nbytes),
                             ctypes.byref(plan), None) == lw.LW_EINVAL        # no field term
    assert lib.lw_batch_deposit(ctypes.byref(lw.lw_batch()), None) == lw.LW_EINVAL

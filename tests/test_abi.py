"""The C-ABI library builds, loads without a GPU, and exports every entry point
that include/blr.h declares.  Host-side argument validation is exercised too
(it returns before any CUDA call).  No compute calls: these run on the CPU."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "blr.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(blr_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1807_05117_gb300.build import build_library
    path = build_library()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path_calls():
    names = _declared()
    for want in ["blr_expand", "blr_project", "blr_state", "blr_adjoint", "blr_gradient",
                 "blr_hessvec", "blr_pcg", "blr_newton"]:
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    from paper_1807_05117_gb300 import blr
    assert sorted(blr.EXPORTED) == _declared()


def test_strerror_and_invalid_params(lib):
    from paper_1807_05117_gb300 import blr
    assert blr.blr_strerror(blr.BLR_ECFL).startswith("displacement")
    bad = [
        dict(n=(16, 16, 16), band=(5, 4, 4)),         # odd band
        dict(n=(16, 16, 16), band=(4, 18, 4)),        # band above the grid
        dict(n=(16, 16, 16), band=(4, 4, 4), nt=0),   # no time step
        dict(n=(16, 16, 16), band=(4, 4, 4), sigma=0.0),
        dict(n=(0, 16, 16), band=(4, 4, 4)),
        dict(n=(16, 16, 16), band=(4, 4, 4), s=0.3),  # 2s not an integer
        dict(n=(16, 16, 16), band=(4, 4, 4), s=-0.5),
        dict(n=(65536, 2, 2), band=(4, 2, 2)),           # x1 planes past the grid limit
    ]
    for kw in bad:
        p = blr.make_params(**{"nt": 4, **kw})
        h = ctypes.c_void_p()
        assert lib.blr_plan_create(ctypes.byref(p), ctypes.byref(h)) == blr.BLR_EINVAL
        assert not h.value
    p = blr.make_params((16, 16, 16), (4, 4, 4))
    p.ckpt_every = -1
    h = ctypes.c_void_p()
    assert lib.blr_plan_create(ctypes.byref(p), ctypes.byref(h)) == blr.BLR_EINVAL
    p = blr.make_params((16, 16, 16), (4, 4, 4))
    p.incompressible = 2
    assert lib.blr_plan_create(ctypes.byref(p), ctypes.byref(h)) == blr.BLR_EINVAL
    p = blr.make_params((16, 16, 16), (4, 4, 4))
    p.hessian = 2
    assert lib.blr_plan_create(ctypes.byref(p), ctypes.byref(h)) == blr.BLR_EINVAL
    # the full Hessian is built for stationary velocities
    p = blr.make_params((16, 16, 16), (4, 4, 4), nonstationary=True, hessian=blr.BLR_NEWTON)
    assert lib.blr_plan_create(ctypes.byref(p), ctypes.byref(h)) == blr.BLR_EINVAL
    p = blr.make_params((16, 16, 16), (4, 4, 4))
    p.nonstationary = 2
    assert lib.blr_plan_create(ctypes.byref(p), ctypes.byref(h)) == blr.BLR_EINVAL
    # the deformation state equation: stationary, no checkpoints
    for kw in (dict(nonstationary=True), dict(nt=4, ckpt_every=2),
               dict(nt=4, ckpt_every=2, hessian=blr.BLR_NEWTON)):
        p = blr.make_params((16, 16, 16), (4, 4, 4),
                            **{"state_equation": blr.BLR_STATE_DEFORMATION, **kw})
        assert lib.blr_plan_create(ctypes.byref(p), ctypes.byref(h)) == blr.BLR_EINVAL
    p = blr.make_params((16, 16, 16), (4, 4, 4))
    p.state_equation = 2
    assert lib.blr_plan_create(ctypes.byref(p), ctypes.byref(h)) == blr.BLR_EINVAL
    # the full Hessian keeps every state: no checkpoints
    p = blr.make_params((16, 16, 16), (4, 4, 4), nt=4, ckpt_every=2, hessian=blr.BLR_NEWTON)
    assert lib.blr_plan_create(ctypes.byref(p), ctypes.byref(h)) == blr.BLR_EINVAL
    # batches take neither the incompressible form, mixed precision nor the full Hessian
    for kw in (dict(incompressible=True), dict(precision=blr.BLR_MIXED),
               dict(hessian=blr.BLR_NEWTON), dict(nonstationary=True),
               dict(state_equation=blr.BLR_STATE_DEFORMATION)):
        arr = (blr.blr_params * 2)(blr.make_params((16, 16, 16), (4, 4, 4), nt=4),
                                   blr.make_params((16, 16, 16), (4, 4, 4), nt=4, **kw))
        assert lib.blr_batch_create(arr, 2, ctypes.byref(h)) == blr.BLR_EINVAL
        assert not h.value
    # NULL plan handles are rejected, destroy(NULL) is a no-op
    assert lib.blr_plan_destroy(None) == blr.BLR_OK
    assert lib.blr_expand(None, None, None, None) == blr.BLR_EINVAL
    assert lib.blr_hessvec(None, None, None, None) == blr.BLR_EINVAL
    vals = (ctypes.c_int * 9)()
    assert lib.blr_plan_tuning(None, vals, 9) == blr.BLR_EINVAL


def test_params_struct_layout_matches_header(tmp_path):
    """The ctypes mirror of blr_params has the size and field offsets that a C
    compiler gives the header's struct (a host C program prints them)."""
    import shutil
    import subprocess
    from paper_1807_05117_gb300 import blr
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = [f for f, _ in blr.blr_params._fields_]
    prog = tmp_path / "layout.c"
    prog.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "blr.h"\nint main(void) {\n'
        '  printf("%zu\\n", sizeof(blr_params));\n'
        + "".join(f'  printf("%zu\\n", offsetof(blr_params, {f}));\n' for f in fields)
        + "  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(prog), "-o", str(exe)],
                   check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    want = [ctypes.sizeof(blr.blr_params)] + [getattr(blr.blr_params, f).offset for f in fields]
    assert got == want


def test_header_compiles_as_c_and_cpp(tmp_path):
    """include/blr.h is plain C (C99) and C++ with the extern "C" guard: both
    compilers accept a translation unit that takes the address of every entry
    point the header declares."""
    import shutil
    import subprocess
    names = _declared()
    body = "".join(f"  (void)&{n};\n" for n in names)
    for cc, ext, std in ((shutil.which("gcc"), "c", "-std=c99"), (shutil.which("g++"), "cpp", "-std=c++17")):
        if cc is None:
            continue
        src_file = tmp_path / f"uses.{ext}"
        src_file.write_text('#include "blr.h"\nvoid uses(void) {\n' + body + "}\n")
        subprocess.run([cc, std, "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), "-c",
                        str(src_file), "-o", str(tmp_path / f"uses_{ext}.o")], check=True)


def test_binding_checks_sizes_and_devices_before_calling(lib):  # noqa: ARG001 (builds the library)
    """The C entry points take bare pointers, so the binding checks element
    counts (from the plan's grid and band), dtypes and devices first: a wrongly
    sized tensor raises ValueError and never reaches the library."""
    import torch

    from paper_1807_05117_gb300 import blr
    sh = blr._shape_of(blr.make_params((8, 6, 4), (4, 2, 4), nt=3, nonstationary=True), 0)
    assert (sh.V, sh.coef, sh.nvel, sh.param) == (192, 96, 3, 288)
    fake = 0x1234
    blr._SHAPES[fake] = sh
    try:
        good = torch.zeros(192 * 3, dtype=torch.float32)
        with pytest.raises(ValueError, match="elements"):
            blr.blr_expand(fake, torch.zeros(95, dtype=torch.complex64), good)
        with pytest.raises(ValueError, match="elements"):
            blr.blr_project(fake, good[:-1], torch.zeros(96, dtype=torch.complex64))
        with pytest.raises(ValueError, match="complex64"):
            blr.blr_gradient(fake, torch.zeros(288, dtype=torch.complex128),
                             torch.zeros(288, dtype=torch.complex64))
        with pytest.raises(ValueError, match="elements"):   # one velocity, not nt
            blr.blr_hessvec(fake, torch.zeros(96, dtype=torch.complex64),
                            torch.zeros(96, dtype=torch.complex64))
        with pytest.raises(ValueError, match="elements"):   # nt body forces
            blr.blr_adjoint(fake, good)
        with pytest.raises(ValueError, match="CUDA tensor"):  # right size, host memory
            blr.blr_project(fake, good, torch.zeros(96, dtype=torch.complex64))
    finally:
        del blr._SHAPES[fake]
    with pytest.raises(ValueError, match="live plan"):
        blr.blr_expand(fake, torch.zeros(96, dtype=torch.complex64), good)

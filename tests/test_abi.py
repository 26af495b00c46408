"""Host-side checks of the C ABI (no GPU needed): the library loads and exports every function
declared in include/parabolic.h, and the binding's struct layouts match the header."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "parabolic.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"PB_API\s+[\w\s\*]+?\b(\w+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_2403_01004_gb300 as pb
    from paper_2403_01004_gb300.build import build
    build()
    return pb.load_library()


def test_library_exports_every_declared_function(lib):
    names = _declared()
    assert len(names) >= 11
    for n in names:
        assert hasattr(lib, n), n
    import paper_2403_01004_gb300 as pb
    assert sorted(pb.EXPORTS) == names
    out = subprocess.run(["nm", "-D", "--defined-only", os.path.join(ROOT, "paper_2403_01004_gb300", "lib",
                                                                    "libparabolic.so")],
                         capture_output=True, text=True).stdout
    exported = {l.split()[-1] for l in out.splitlines() if " T " in l}
    assert set(names) <= exported


def test_struct_layouts_match_header(tmp_path):
    """Compiles a tiny C program against the header and compares sizeof/offsetof with ctypes."""
    import paper_2403_01004_gb300 as pb
    prog = tmp_path / "layout.c"
    fields = {
        "pb_grid": ("PbGrid", ["n_r", "n_theta", "n_phi", "r_face", "t_face"]),
        "pb_operator": ("PbOperator", ["kind", "C", "T0", "n", "B", "rho", "nu"]),
        "pb_advance_opts": ("PbAdvanceOpts", ["scheme", "use_ptl", "max_cycles", "ptl_floor", "dt_cycles",
                                              "n_forced", "rtol", "max_iter", "fixed_iters", "check_every",
                                              "judge_guess", "mixed_precision", "inner_rtol", "ptl_mode",
                                              "precond", "pc_degree"]),
        "pb_train_opts": ("PbTrainOpts", ["steps", "batch", "crop", "border", "lr", "seed"]),
        "pb_tune": ("PbTune", ["kchunk", "blocks_per_sm", "small_tiles"]),
        "pb_kernel_stat": ("PbKernelStat", ["name", "launches", "timed_launches", "total_ms", "bytes"]),
        "pb_stats": ("PbStats", ["cycles", "status_cycle", "total_stages", "total_iters", "dt_explicit",
                                 "last_dt_ptl", "fmax", "k_index", "final_rel_residual", "cycle_capacity",
                                 "dt_cycle", "work_cycle", "dt_ptl_cycle", "k_cycle", "guess_used"]),
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', f'#include "{HEADER}"', "int main(void) {"]
    for cname, (_, fl) in fields.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f in fl:
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    prog.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", str(prog), "-o", str(exe)], check=True)
    got = dict(l.rsplit(" ", 1) for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.splitlines())
    for cname, (pyname, fl) in fields.items():
        cls = getattr(pb, pyname)
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f in fl:
            assert int(got[f"{cname}.{f}"]) == getattr(cls, f).offset, (cname, f)


def test_status_strings_and_defaults(lib):
    import paper_2403_01004_gb300 as pb
    assert lib.pb_status_string(0).decode() == "ok"
    assert "converge" in lib.pb_status_string(pb.PB_ENOCONVERGE).decode()
    o = pb.PbAdvanceOpts()
    lib.pb_advance_opts_init(ctypes.byref(o))
    assert o.use_ptl == 1 and o.ptl_floor == 1.0 and o.rtol == 1e-10 and o.max_cycles == 100000


def test_setup_rejects_bad_grid_without_touching_the_gpu(lib):
    import paper_2403_01004_gb300 as pb
    rf = (ctypes.c_double * 2)(1.0, 2.0)
    tf = (ctypes.c_double * 3)(0.0, 1.0, 2.0)
    g = pb.PbGrid(1, 2, 4, ctypes.cast(rf, ctypes.POINTER(ctypes.c_double)),
                  ctypes.cast(tf, ctypes.POINTER(ctypes.c_double)))
    op = pb.PbOperator()
    h = ctypes.c_void_p()
    rc = lib.parabolic_setup(ctypes.byref(g), ctypes.byref(op), 0, None, ctypes.byref(h))
    assert rc == pb.PB_EINVAL
    assert b"n_r" in lib.pb_last_error(None)

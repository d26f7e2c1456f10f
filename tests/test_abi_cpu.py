"""CPU checks of the C ABI: the library builds for sm_103a, loads without a GPU,
exports every function include/hqa.h declares, and the ctypes structures have
the C layout (checked against a host program compiled from the header)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hqa.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2004_03972_gb300 import build, hqa
    build.build()
    return hqa.lib()


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(?:hqa_status|void|const char\s*\*)\s+(hqa_\w+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(lib, n), n
    from paper_2004_03972_gb300 import hqa
    assert sorted(hqa.EXPORTS) == names


def test_status_strings_and_defaults(lib):
    from paper_2004_03972_gb300 import hqa
    for code in range(10):
        assert lib.hqa_status_string(code)
    s = hqa.schedule()
    assert (s.kind, s.alpha_f, s.rho1, s.rho2) == (0, 0.008, 4.0, 3.0)
    assert (s.beta_f, s.kappa1, s.kappa2, s.M, s.hstep, s.window) == (0.12, 0.05, 1.0, 6, 1.0, 100)


def test_struct_layout_matches_header(tmp_path):
    import ctypes as C
    from paper_2004_03972_gb300 import hqa
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "hqa.h"\n'
        "#define P(T, f) printf(#T \" \" #f \" %zu\\n\", offsetof(T, f));\n"
        "int main(void) {\n"
        " printf(\"hqa_schedule size %zu\\n\", sizeof(hqa_schedule));\n"
        " printf(\"hqa_run_opts size %zu\\n\", sizeof(hqa_run_opts));\n"
        " printf(\"hqa_result size %zu\\n\", sizeof(hqa_result));\n"
        " printf(\"hqa_plan_info size %zu\\n\", sizeof(hqa_plan_info));\n"
        " printf(\"hqa_tune_entry size %zu\\n\", sizeof(hqa_tune_entry));\n"
        + "".join(f" P(hqa_schedule, {f})\n" for f, _ in hqa.Schedule._fields_)
        + "".join(f" P(hqa_run_opts, {f})\n" for f, _ in hqa.RunOpts._fields_)
        + "".join(f" P(hqa_result, {f})\n" for f, _ in hqa.Result._fields_)
        + "".join(f" P(hqa_plan_info, {f})\n" for f, _ in hqa.PlanInfo._fields_)
        + "".join(f" P(hqa_tune_entry, {f})\n" for f, _ in hqa.TuneEntry._fields_)
        + " return 0; }\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    table = {"hqa_schedule": hqa.Schedule, "hqa_run_opts": hqa.RunOpts, "hqa_result": hqa.Result,
             "hqa_plan_info": hqa.PlanInfo, "hqa_tune_entry": hqa.TuneEntry}
    for line in got:
        if not line:
            continue
        t, f, v = line.split()
        if f == "size":
            assert C.sizeof(table[t]) == int(v), t
        else:
            assert getattr(table[t], f).offset == int(v), (t, f)


def test_enum_constants_match_header(tmp_path):
    """The binding's constants equal the header's enumerators (a host program
    compiled from include/hqa.h prints them)."""
    from paper_2004_03972_gb300 import hqa
    pairs = {f"HQA_{k}": v for k, v in (
        ("SCHED_PAPER", hqa.SCHED_PAPER), ("SCHED_LINEAR_GAMMA", hqa.SCHED_LINEAR_GAMMA),
        ("SCHED_TABLE", hqa.SCHED_TABLE), ("INIT_PAPER", hqa.INIT_PAPER),
        ("INIT_RANDOM_FLUX", hqa.INIT_RANDOM_FLUX), ("INIT_GIVEN", hqa.INIT_GIVEN),
        ("PREC_FP32", hqa.PREC_FP32), ("PREC_BF16", hqa.PREC_BF16),
        ("PREC_BF16X2", hqa.PREC_BF16X2), ("PREC_FP16", hqa.PREC_FP16),
        ("PREC_FP16X2", hqa.PREC_FP16X2), ("J_BF16", hqa.J_BF16), ("J_FP16", hqa.J_FP16),
        ("J_FP32", hqa.J_FP32), ("J_FP8", hqa.J_FP8), ("KERNEL_AUTO", hqa.KERNEL_AUTO),
        ("KERNEL_SCALAR", hqa.KERNEL_SCALAR), ("KERNEL_VECTOR", hqa.KERNEL_VECTOR),
        ("KERNEL_DENSE", hqa.KERNEL_DENSE), ("KERNEL_LOWDEG", hqa.KERNEL_LOWDEG),
        ("KERNEL_STREAM", hqa.KERNEL_STREAM),
        ("MLP_IN", hqa.MLP_IN), ("MLP_HIDDEN", hqa.MLP_HIDDEN), ("MLP_OUT", hqa.MLP_OUT),
        ("MLP_PARAMS", hqa.MLP_PARAMS))}
    pairs.update({name: code for code, name in hqa.STATUS_NAMES.items()})
    src = tmp_path / "enums.c"
    src.write_text('#include <stdio.h>\n#include "hqa.h"\nint main(void) {\n'
                   + "".join(f' printf("{n} %d\\n", (int)({n}));\n' for n in pairs)
                   + " return 0; }\n")
    exe = tmp_path / "enums"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    values = dict(zip(got[0::2], map(int, got[1::2])))
    assert values == pairs


def test_library_has_no_cuda_runtime_dependency(lib):
    from paper_2004_03972_gb300 import hqa
    out = subprocess.run(["ldd", hqa.LIB_PATH], capture_output=True, text=True).stdout
    assert "libcudart" not in out   # static runtime: loads on hosts without the toolkit


def test_product_path_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_2004_03972_gb300 import hqa
    monkeypatch.setattr(hqa, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(hqa, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        hqa.lib()

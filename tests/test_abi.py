"""Host-side checks of the C ABI: the library builds, loads, and exports every
entry point declared in include/cwb.h (no GPU work is issued)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(cwb_[a-z_0-9]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2110_03513_gb300 import binding
    return ctypes.CDLL(binding.library_path())


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("cwb_create", "cwb_fit", "cwb_predict", "cwb_free", "cwb_get_coefficients", "cwb_get_trace",
                     "cwb_get_fitted", "cwb_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2110_03513_gb300 import binding
    missing = [n for n in sorted(_declared()) if n not in binding._SIGS]
    assert not missing, missing


def test_null_and_invalid_arguments_fail_without_gpu(lib):
    from paper_2110_03513_gb300 import binding
    L = binding.load_library()
    out = ctypes.c_void_p(123)
    st = L.cwb_create(None, None, 0, 10, 1, None, None, None, 1, 0, ctypes.byref(out))
    assert st == 1 and out.value is None
    assert "NULL" in binding.cwb_last_error()
    L.cwb_free(None)          # NULL-safe
    assert L.cwb_fit(None, 5) == 1


def test_binding_structs_match_the_header_layout(tmp_path):
    """The ctypes structs of the binding have the C compiler's size and field offsets for every
    struct include/cwb.h declares (compiled here with gcc as plain C)."""
    import subprocess
    from paper_2110_03513_gb300 import binding
    structs = {name: getattr(binding, name) for name in ("cwb_learner", "cwb_config", "cwb_learner_info",
                                                          "cwb_server_config", "cwb_shard_config",
                                                          "cwb_fit_request")}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cwb.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            cname = {"lam": "lambda", "lam_full": "lambda_full"}.get(field, field)
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {cname}));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_noalloc_size_check_rejects_wrapping_requests(tmp_path):
    """The size check of cwb_predict_noalloc (host code, compiled here as plain C): requests whose
    byte counts would wrap around 64 bits are rejected before any product is formed, the largest
    request that fits is accepted with the exact byte count, and one more row is rejected."""
    import subprocess
    limit = 16 << 20
    src = tmp_path / "need.c"
    src.write_text("\n".join([
        "#include <stdio.h>",
        "#include <inttypes.h>",
        '#include "cwb_noalloc_size.h"',
        "int main(int argc, char** argv) {",
        "  const int64_t cases[][3] = {",
        "    {INT64_C(1) << 62, 50, 4}, {INT64_C(1) << 61, 3, 8}, {INT64_MAX, 1, 4}, {INT64_C(1) << 40, 1, 4},",
        "    {0, 7, 4}, {1, 7, 8}, {-1, 3, 4}, {5, 0, 4}, {5, 3, 2},",
        f"    {{({limit} - 255) / (4 * 50 + 4), 50, 4}}, {{({limit} - 255) / (4 * 50 + 4) + 1, 50, 4}},",
        f"    {{({limit} - 255) / (8 * 3 + 4), 3, 8}}, {{({limit} - 255) / (8 * 3 + 4) + 1, 3, 8}}}};",
        "  for (unsigned i = 0; i < sizeof cases / sizeof cases[0]; ++i) {",
        "    uint64_t need = 0;",
        f"    int ok = cwb_noalloc_need(cases[i][0], cases[i][1], cases[i][2], {limit}u, &need);",
        '    printf("%d %" PRIu64 "\\n", ok, need);',
        "  }",
        "  return 0; }"]))
    exe = tmp_path / "need"
    subprocess.check_call(["gcc", "-std=c11", "-Wall", "-Werror", "-I",
                           os.path.join(ROOT, "paper_2110_03513_gb300", "csrc"), str(src), "-o", str(exe)])
    rows = [tuple(int(v) for v in l.split()) for l in subprocess.check_output([str(exe)], text=True).split("\n")
            if l.strip()]
    ok = [r[0] for r in rows]
    assert ok == [0, 0, 0, 0, 1, 1, 0, 0, 0, 1, 0, 1, 0]
    assert rows[4][1] == 0                                  # no rows: nothing staged
    assert rows[5][1] == 256 + 4                            # one row of 7 FP64 values: 56 -> 256, + 4
    for i, (p, xsz) in ((9, (50, 4)), (11, (3, 8))):
        n_new = (limit - 255) // (xsz * p + 4)
        want = -(-xsz * p * n_new // 256) * 256 + 4 * n_new
        assert rows[i][1] == want <= limit

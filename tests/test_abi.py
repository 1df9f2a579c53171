"""C-ABI library: builds, loads and exports every symbol include/*.h declares
(no compute calls: these run without a GPU)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(ngs_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2603_16103_gb300 import build
    return ctypes.CDLL(build.build())


def test_header_declares_the_pass_api():
    names = declared_functions()
    for required in ("ngs_build_graph", "ngs_edge_costs", "ngs_select_pairs",
                     "ngs_merge_compact", "ngs_simplify"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2603_16103_gb300 import binding
    missing = [n for n in declared_functions() if n not in binding._SIGS]
    assert not missing, missing


def test_default_params_host_only():
    from paper_2603_16103_gb300 import binding
    p = binding.ngs_default_params()
    assert (p.k, p.mc_samples, p.cost_mode, p.max_passes, p.prefilter) == (16, 1, 0, 64, 1)
    assert abs(p.tau - 0.005) < 1e-15 and p.eig_floor == 1e-30
    assert p.lambda_geo == 1.0 and p.lambda_app == 1.0


def test_struct_layouts_match_header():
    """ctypes mirrors of the C structs have the C sizes (checked with gcc)."""
    import subprocess
    import tempfile
    from paper_2603_16103_gb300 import binding
    names = ["ngs_splats", "ngs_params", "ngs_graph", "ngs_stats", "ngs_server_config",
             "ngs_job_info", "ngs_server_stats", "ngs_tuning"]
    src = ('#include <stdio.h>\n#include "ngs.h"\nint main(){'
           + "".join(f'printf("%zu\\n", sizeof({n}));' for n in names) + "}\n")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "s.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "s")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        sizes = [int(x) for x in subprocess.run([exe], capture_output=True, text=True,
                                                check=True).stdout.split()]
    assert sizes == [ctypes.sizeof(getattr(binding, n)) for n in names]


def test_binding_constants_match_header():
    """Status codes and limits of the binding equal the header's macros (gcc)."""
    import subprocess
    import tempfile
    from paper_2603_16103_gb300 import binding
    names = ["NGS_OK", "NGS_ERR_INVALID_ARG", "NGS_ERR_OOM", "NGS_ERR_CUDA", "NGS_ERR_TIMEOUT",
             "NGS_ERR_BUDGET", "NGS_ERR_STATE", "NGS_MAX_K", "NGS_MAX_N", "NGS_MAX_S",
             "NGS_MAX_SCENES", "NGS_STATS_MAX_PASSES"]
    src = ('#include <stdio.h>\n#include "ngs.h"\nint main(){'
           + "".join(f'printf("%lld\\n", (long long)({n}));' for n in names) + "}\n")
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "k.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "k")
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        vals = [int(x) for x in subprocess.run([exe], capture_output=True, text=True,
                                               check=True).stdout.split()]
    assert vals == [getattr(binding, n) for n in names]


def test_default_tuning_host_only():
    from paper_2603_16103_gb300 import binding
    t = binding.ngs_default_tuning()
    assert (t.knn_block_min, t.cells_per_point, t.cost_blocks_per_sm, t.match_method,
            t.match_max_steps, t.scan_method, t.wait_test_tile) == (64, 4, 8, 2, 65536, 0, -1)


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2603_16103_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True) + \
            glob.glob(os.path.join(pkg, "csrc", "*")):
        text = open(f, errors="replace").read()
        assert "import oracle" not in text and "from oracle" not in text, f
        assert "ngs_oracle" not in text and "liboracle" not in text, f

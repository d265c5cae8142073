"""CPU checks of the C ABI: the library builds for sm_103a, loads, and exports every
function that include/*.h declares (no compute calls: there is no GPU here)."""
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
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(gpfc_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gpfc_create", "gpfc_destroy", "gpfc_fold", "gpfc_score_box", "gpfc_search",
                     "gpfc_best_period", "gpfc_sync", "gpfc_strerror"):
        assert required in names


def test_library_loads_and_exports_every_declared_symbol():
    import paper_2312_02063_gb300 as g
    lib = g.load_library()
    missing = [n for n in sorted(declared_functions()) if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    import paper_2312_02063_gb300 as g
    lib = g.load_library()
    assert lib.gpfc_strerror(0) == b"ok"
    assert lib.gpfc_strerror(-4) == b"value outside the fixed-point range"
    assert lib.gpfc_version() >= 100


def test_null_context_is_rejected_without_gpu():
    import paper_2312_02063_gb300 as g
    lib = g.load_library()
    assert lib.gpfc_sync(None) == -1
    assert lib.gpfc_fold(None, None, None, 0, None, 0, 64, 0.0, None, None) == -1


def test_product_path_has_no_cpu_fallback():
    import torch
    import paper_2312_02063_gb300 as g
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(g.GpfcError):
        g.Context(0)


def test_product_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2312_02063_gb300")
    for f in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if f.endswith((".py", ".cu", ".cuh", ".h")):
            text = open(f).read()
            assert "import oracle" not in text and "from oracle" not in text, f
            assert "gpfc_oracle" not in text, f


def test_sm103a_binary_is_built():
    import paper_2312_02063_gb300 as g
    g.load_library()
    logs = glob.glob(os.path.join(ROOT, "paper_2312_02063_gb300", "_build", "*.ptxas.txt"))
    assert logs and any("sm_103a" in open(l).read() for l in logs)


def test_struct_layouts_match_the_header(tmp_path):
    """sizeof / offsetof of the public structs, compiled from include/gpfc.h with gcc, equal
    the ctypes mirrors the Python binding passes across the boundary."""
    import shutil
    import subprocess
    import paper_2312_02063_gb300 as g
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stddef.h>\n#include <stdio.h>\n#include "gpfc.h"\n'
        'int main(void) {\n'
        '  printf("%zu %zu %zu %zu %zu %zu %d %d %d %d %d %d\\n", sizeof(gpfc_fold_config),\n'
        '         sizeof(gpfc_box_params), sizeof(gpfc_cnn_weights),\n'
        '         offsetof(gpfc_fold_config, blocks_per_sm), sizeof(gpfc_star_summary), sizeof(gpfc_peak),\n'
        '         (int)GPFC_BOX_AUTO, (int)GPFC_BOX_EPILOGUE, (int)GPFC_BOX_WARP, (int)GPFC_BOX_FUSED,\n'
        '         (int)GPFC_SCORER_BOX, (int)GPFC_SCORER_CNN);\n'
        '  return 0;\n}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert int(out[0]) == ctypes.sizeof(g.FoldConfig)
    assert int(out[1]) == ctypes.sizeof(g.BoxParams)
    assert int(out[2]) == ctypes.sizeof(g.CnnWeights)
    assert int(out[3]) == g.FoldConfig.blocks_per_sm.offset
    assert [int(v) for v in out[6:12]] == [g.BOX_AUTO, g.BOX_EPILOGUE, g.BOX_WARP, g.BOX_FUSED, g.SCORER_BOX,
                                           g.SCORER_CNN]
    assert int(out[4]) == g.STAR_SUMMARY_DTYPE.itemsize
    src2 = tmp_path / "layout2.c"
    src2.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "gpfc.h"\nint main(void) { printf("%zu %zu\\n", '
                    'sizeof(gpfc_detrend_params), offsetof(gpfc_detrend_params, spacings)); return 0; }\n')
    exe2 = tmp_path / "layout2"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src2), "-o", str(exe2)], check=True)
    o2 = subprocess.run([str(exe2)], check=True, capture_output=True, text=True).stdout.split()
    assert int(o2[0]) == ctypes.sizeof(g.DetrendParams) and int(o2[1]) == g.DetrendParams.spacings.offset
    assert int(out[5]) == g.PEAK_DTYPE.itemsize


def test_batched_entry_rejects_null_context_without_gpu():
    import paper_2312_02063_gb300 as g
    lib = g.load_library()
    assert lib.gpfc_search_batched(None, 1, None, None, None, 1, None, None, 1, None, 64, 0, None, None, None,
                                   None) == -1
    assert lib.gpfc_set_graph(None, 1) == -1
    assert lib.gpfc_set_autotune(None, 1) == -1
    assert lib.gpfc_check_wait_timeout(None, 10000) == -1
    assert lib.gpfc_peaks(None, None, None, 1, None, 1, 3.0, 4, 1e-3, 8, None, None) == -1
    assert lib.gpfc_fold_equal_count(None, None, None, 1, None, 1, 4096, 256, 0.0, None) == -1
    assert lib.gpfc_set_box_path(None, g.BOX_FUSED) == -1
    import ctypes
    ms, nl = ctypes.c_float(), ctypes.c_int32()
    assert lib.gpfc_fold_launch_times(None, ctypes.byref(ms), ctypes.byref(nl)) == -1



def test_noalloc_entry_rejects_bad_arguments_without_gpu():
    """gpfc_best_period_noalloc checks its arguments before any CUDA call, so the
    rejections run here with fake (never dereferenced) device pointers."""
    import ctypes
    import paper_2312_02063_gb300 as g
    lib = g.load_library()
    fake = ctypes.c_void_p(0x1000)
    f = lib.gpfc_best_period_noalloc
    assert f(None, 10, fake, fake, None) == -1           # no score
    assert f(fake, 10, None, None, None) == -1           # both outputs NULL
    assert f(fake, 0, fake, fake, None) == -1            # empty
    assert f(fake, -5, fake, None, None) == -1           # negative size
    assert f(fake, 2 ** 31, fake, None, None) == -1      # beyond the 32-bit index of the key
    assert f(fake, 2 ** 40, None, fake, None) == -1


def test_smem_probe_rejects_bad_arguments_without_gpu():
    import paper_2312_02063_gb300 as g
    lib = g.load_library()
    f = lib.gpfc_probe_smem_rmw
    assert f(5, 0, 32, 16, 1, 100, None, None, None) == -1      # word size
    assert f(8, 2, 32, 16, 1, 100, None, None, None) == -1      # operation
    assert f(8, 0, 48, 16, 1, 100, None, None, None) == -1      # not a power of two
    assert f(8, 1, 32, 0, 1, 100, None, None, None) == -1       # no warps
    assert f(4, 0, 32, 16, 1, 0, None, None, None) == -1        # no iterations


def test_detrend_rejects_bad_arguments_without_gpu():
    import paper_2312_02063_gb300 as g
    lib = g.load_library()
    assert lib.gpfc_detrend(None, None, None, None, 10, None, None, None, None, None) == -1

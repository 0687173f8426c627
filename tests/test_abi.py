"""The C-ABI library builds, loads without a GPU and exports every entry point
that include/recon.h declares; the binding mirrors them.  No GPU."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "recon.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(recon_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2401_01404_gb300 import build

    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["recon_init", "recon_best_pairs", "recon_score", "recon_cd_sweep", "recon_objective",
              "recon_get_model", "recon_save", "recon_load", "recon_last_error", "recon_destroy"]:
        assert n in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (recon_[a-z_]+)\b", out))
    missing = [n for n in _declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_binding_covers_the_header(libpath):
    from paper_2401_01404_gb300 import recon

    L = recon.lib()
    for n in _declared():
        assert hasattr(L, n)
        assert n in recon._EXPORTS, n
    assert hasattr(recon, "recon_init") and hasattr(recon, "recon_best_pairs")


def test_default_options_without_a_gpu(libpath):
    from paper_2401_01404_gb300 import recon

    o = recon.recon_default_options()
    assert o.seed == 1 and abs(o.eps_knn - 1e-3) < 1e-15 and o.h_clamp == 10.0
    assert o.knn_mode == recon.RECON_KNN_NNDESCENT


def test_init_fails_loudly_without_a_gpu(libpath):
    """There is no CPU fallback: on a machine without a usable GPU, recon_init
    returns an error instead of computing anything."""
    import numpy as np
    import torch

    from paper_2401_01404_gb300 import recon

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(recon.ReconError) as e:
        recon.recon_init(np.ones((4, 3), dtype=np.int8))
    assert e.value.status in (recon.RECON_ECUDA, recon.RECON_ENOMEM)


def test_argument_errors_without_a_gpu(libpath):
    import numpy as np

    from paper_2401_01404_gb300 import recon

    with pytest.raises(recon.ReconError) as e:
        recon.recon_init(np.ones((4, 1), dtype=np.int8))  # N = 1
    assert e.value.status == recon.RECON_EINVAL
    with pytest.raises(recon.ReconError) as e:
        recon.recon_init(np.ones((4, 3), dtype=np.float32), recon.RECON_ISING)
    assert e.value.status == recon.RECON_EINVAL
    with pytest.raises(recon.ReconError) as e:
        recon.recon_init(np.ones((4, 3), dtype=np.int8), options=recon.recon_default_options(lam=-1.0))
    assert e.value.status == recon.RECON_EINVAL


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures (options, statistics, device ceilings,
    training options) have the header's size and field offsets: a field added on
    one side only would shift every later field silently.  Checked by compiling
    a small C program against include/recon.h with the host compiler."""
    import ctypes
    import shutil

    from paper_2401_01404_gb300 import recon as R

    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no host C compiler")
    structs = {"recon_options": R.recon_options, "recon_stats": R.recon_stats, "recon_peaks": R.recon_peaks,
               "recon_train_opts": R.recon_train_opts}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "recon.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append(f'    printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            cfield = fname.rstrip("_")  # (lambda_ in Python is lambda in C)
            lines.append(f'    printf("{cname}.{fname} %zu\\n", offsetof({cname}, {cfield}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                               check=True).stdout.splitlines())
    for cname, cls in structs.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(cls, fname).offset, (cname, fname)

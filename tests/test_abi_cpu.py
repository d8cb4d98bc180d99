"""The C-ABI library loads and exports every declared symbol (no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "phoebe_gpu.h")).read()
    return sorted(set(re.findall(r"\b(phoebe_gpu_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    import paper_2111_14999_b300 as pg
    lib = ctypes.CDLL(pg.LIB_PATH)
    declared = _declared()
    assert len(declared) >= 15
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(pg.EXPORTED) == sorted(declared)


def test_constants_match_oracle_literals():
    # the library and the oracle carry the physical constants as independent literals
    import paper_2111_14999_b300 as pg
    from oracle import elph
    kb, hw, zp = pg.constants()
    assert kb == elph.KB_EV and hw == elph.HBAR_OMEGA_EV and zp == elph.HBAR2_AMU_EV_A2


def test_params_struct_defaults_and_layout():
    import paper_2111_14999_b300 as pg
    from workloads import synthetic as W
    s = pg.make_params(W.toy()[1], k_subset=[1, 2, 5])
    assert list(s.nk) == [8, 8, 8] and s.delta_cut_sigmas == 6.0 and s.omega_cut_eV == 1e-4
    assert s.n_k_subset == 3 and s.k_subset[2] == 5
    assert s.sampler == 0 and s.sample_fraction == 0.05 and s.mix_alpha == 0.1
    o = pg.binding.TrainOpts()
    pg.lib.phoebe_gpu_train_opts_default(ctypes.byref(o))
    assert o.epochs > 0 and o.states_per_step > 0 and o.lr > 0


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of a header struct, from gcc."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "lay.c"
    body = "".join(f'printf("%zu ", offsetof({struct}, {f}));' for f in fields)
    src.write_text(f'#include <stdio.h>\n#include <stddef.h>\n#include "phoebe_gpu.h"\n'
                   f'int main(void){{printf("%zu ", sizeof({struct}));{body}return 0;}}\n')
    exe = tmp_path / "lay"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    return [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()]


def test_ctypes_structs_mirror_the_header(tmp_path):
    import paper_2111_14999_b300 as pg
    for py, cname in ((pg.RTAParams, "phoebe_gpu_rta_params"), (pg.binding.Stats, "phoebe_gpu_stats"),
                      (pg.binding.TrainOpts, "phoebe_gpu_train_opts"),
                      (pg.binding.BatchOpts, "phoebe_gpu_batch_opts")):
        names = [f for f, _ in py._fields_]
        got = _c_layout(cname, names, tmp_path)
        assert got[0] == ctypes.sizeof(py), cname
        assert got[1:] == [getattr(py, f).offset for f in names], cname


def test_create_without_gpu_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2111_14999_b300 as pg
    with pytest.raises(pg.PhoebeGPUError):
        pg.PhoebeGPU(0)
    assert pg.version().startswith("phoebe_gpu")


def test_make_params_carries_every_workload_field():
    # every field of the workloads parameter record reaches the C struct (no silent drop)
    import dataclasses
    from workloads import synthetic as W
    pg = pytest.importorskip("paper_2111_14999_b300")
    prm = W.RTAParams(nk=(4, 4, 4), nq=(8, 8, 8), T_K=250.0, mu_eV=0.3, sigma_eV=0.02, window_eV=0.4,
                      delta_cut_sigmas=5.0, omega_cut_eV=2e-4, degen_tol_eV=1e-7, precision=7,
                      sampler=2, sample_fraction=0.1, mix_alpha=0.2, seed=7, sampler_fp32_network=1,
                      population_delta=0.01, smearing=1, sigma_min_eV=3e-3)
    s = pg.make_params(prm)
    for f in dataclasses.fields(prm):
        v = getattr(prm, f.name)
        if f.name == "k_subset" or v is None:
            continue
        got = getattr(s, f.name)
        if f.name in ("nk", "nq"):
            assert list(got) == list(v), f.name
        else:
            assert got == pytest.approx(v), f.name

"""The Python binding's argument marshalling on the host: the ctypes structures mirror
include/mhd.h field by field, and device-pointer arguments must be contiguous float64 CUDA tensors
(a CPU tensor, another dtype or a strided view is refused before any call reaches the library)."""
import os
import re

import pytest
import torch

import paper_1811_02605_gb300 as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _struct_fields(name):
    src = open(os.path.join(ROOT, "include", "mhd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct\s*\{([^}]*)\}\s*" + name + r"\s*;", src).group(1)
    out = []
    for decl in body.split(";"):
        decl = decl.strip()
        if not decl:
            continue
        names = decl.split(None, 1)[1]
        for n in names.split(","):
            n = n.strip().lstrip("*").strip()
            out.append(re.sub(r"\[.*\]", "", n))
    return out


@pytest.mark.parametrize("cname,pyname", [("mhd_params_t", "Params"), ("mhd_step_info_t", "StepInfo"),
                                           ("mhd_grid_desc_t", "GridDesc"), ("mhd_fields_t", "Fields")])
def test_structures_mirror_the_header(cname, pyname):
    assert [f[0] for f in getattr(P, pyname)._fields_] == _struct_fields(cname)


def test_device_pointer_arguments_are_checked_on_the_host():
    with pytest.raises(TypeError):
        P.make_fields([0.0], [0.0], [0.0])
    with pytest.raises(ValueError):
        P.make_fields(torch.zeros(4, dtype=torch.float64), torch.zeros(4), torch.zeros(4))


def test_make_params_defaults():
    p = P.make_params()
    assert p.precision == P.PREC_FP64 and p.preconditioner == 0 and p.pcg_variant == 0
    assert p.viscosity_sts == 0 and p.resistivity_implicit == 0 and p.mixed_restart == 0
    assert p.tol == 1e-9 and p.alpha_si_fixed < 0

"""The C ABI library loads and exports every symbol include/lbdp.h and
include/lbdp_batch.h declare, and the ctypes structures match the C layout
(no GPU needed: no compute calls are made)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDRS = [os.path.join(ROOT, "include", h) for h in ("lbdp.h", "lbdp_batch.h")]


@pytest.fixture(scope="module")
def built():
    from paper_2202_01631_gb300 import build
    return build.build()


def declared_functions():
    names = set()
    for hdr in HDRS:
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(lb[bs]?_[a-z_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("lb_create", "lb_set_fields", "lb_add_particle", "lb_step", "lb_read_fields",
                 "lb_read_particles", "lb_conservation", "lb_destroy", "lbb_create", "lbb_add_box",
                 "lbb_run", "lbb_tune", "lbs_submit", "lbs_pump", "lbs_poll", "lb_arena_alloc"):
        assert need in names


def test_library_exports_every_declared_symbol(built):
    lib = C.CDLL(built)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (lb[bs]?_[a-z_]+)\b", out))
    assert set(declared_functions()) <= exported


def test_host_only_entry_points(built):
    from paper_2202_01631_gb300 import lbdp
    assert abs(lbdp.lb_wetting_h(90.0)) < 1e-15
    assert abs(lbdp.lb_wetting_h(60.0) - 0.334933) < 1e-6
    assert abs(lbdp.lb_solubility_E(2.0, 1.0) - 0.43768) < 1e-5
    assert lbdp._err_string(-4).startswith("particles")
    p = lbdp.lb_params(nx=32, ny=32, nz=32, precision="fp32")
    assert lbdp.lb_device_bytes(p) > 32 ** 3 * 152
    bad = lbdp.lb_params(nx=0, ny=4, nz=4)
    with pytest.raises(lbdp.LbError):
        lbdp.lb_device_bytes(bad)
    bad_tau = lbdp.lb_params(nx=4, ny=4, nz=4, tau=0.5)
    with pytest.raises(lbdp.LbError):
        lbdp.lb_device_bytes(bad_tau)


def test_struct_layout_matches_header(tmp_path, built):
    from paper_2202_01631_gb300 import lbdp
    src = tmp_path / "layout.c"
    structs = (("lb_params", lbdp.LbParams), ("lb_particle_desc", lbdp.LbParticleDesc),
               ("lb_particle_state", lbdp.LbParticleState), ("lbb_params", lbdp.LbbParams),
               ("lbs_params", lbdp.LbsParams), ("lbs_request", lbdp.LbsRequest),
               ("lbs_result", lbdp.LbsResult))
    fields = {s: [f for f, _ in cls._fields_] for s, cls in structs}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbdp_batch.h"', "int main(void){"]
    for s, fs in fields.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (s, s))
        for f in fs:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (s, f, s, f))
    lines.append("return 0;}")
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True).stdout.split("\n") if l)
    for s, cls in structs:
        assert int(got[s]) == C.sizeof(cls)
        for f, _ in cls._fields_:
            assert int(got["%s.%s" % (s, f)]) == getattr(cls, f).offset, (s, f)

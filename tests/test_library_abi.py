"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
function that include/pp_cweno.h declares."""
import ctypes
import os
import re

import pytest

from paper_1402_5618_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pp_cweno.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pp_cweno_[a-z_]+)\s*\(", src)))


def test_header_matches_binding_list():
    assert _declared() == sorted(binding.EXPORTS)


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_config_struct_layout_matches_header():
    # sizeof(pp_cweno_config) as laid out by the C compiler on this host
    import subprocess
    import tempfile
    src = '#include "pp_cweno.h"\n#include <stdio.h>\n#include <stddef.h>\n' \
          'int main(){printf("%zu %zu %zu %zu %zu\\n", sizeof(pp_cweno_config), ' \
          'sizeof(pp_cweno_stats_t), offsetof(pp_cweno_config, limiter), ' \
          'offsetof(pp_cweno_config, flux), offsetof(pp_cweno_config, recon));return 0;}\n'
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        open(c, "w").write(src)
        exe = os.path.join(d, "t")
        subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    assert int(out[0]) == ctypes.sizeof(binding.Config)
    assert int(out[1]) == ctypes.sizeof(binding.Stats)
    assert int(out[2]) == binding.Config.limiter.offset
    assert int(out[3]) == binding.Config.flux.offset
    assert int(out[4]) == binding.Config.recon.offset


def test_config_rejects_unknown_flux():
    """The configuration check runs before any device call: an unknown flux
    selector is PP_ERR_ARG, for one problem and for a batch whose problems
    disagree on the flux."""
    L = binding.lib()
    h = ctypes.c_void_p()
    for bad in (-1, 2, 99):
        c = binding.make_config(flux=bad)
        assert L.pp_cweno_create(ctypes.byref(c), None, ctypes.byref(h)) == binding.PP_ERR_ARG
        assert not h.value
    arr = (binding.Config * 2)(binding.make_config(flux=binding.FLUX_HLLC),
                               binding.make_config(flux=binding.FLUX_LLF))
    assert L.pp_cweno_create_batch(arr, 2, None, ctypes.byref(h)) == binding.PP_ERR_ARG
    assert not h.value


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    monkeypatch.setattr(build, "LIB", str(tmp_path / "absent.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError):
        binding.lib()


def test_characteristic_form_limits():
    """Reconstruction selectors are checked before any device call: an
    unknown one is PP_ERR_ARG, and so is a batch whose problems mix the
    component-wise and characteristic-wise forms (the allocation-free
    operator's refusal of the characteristic form is checked with real
    device buffers in the GPU tests)."""
    L = binding.lib()
    h = ctypes.c_void_p()
    c = binding.make_config(recon=2)
    assert L.pp_cweno_create(ctypes.byref(c), None, ctypes.byref(h)) == binding.PP_ERR_ARG
    c0 = binding.make_config(recon=binding.RECON_COMPONENT)
    c1 = binding.make_config(recon=binding.RECON_CHARACTERISTIC)
    arr = (binding.Config * 2)(c1, c0)
    assert L.pp_cweno_create_batch(arr, 2, None, ctypes.byref(h)) == binding.PP_ERR_ARG
    assert not h.value

"""The C-ABI library builds, loads and exports every symbol include/smc.h
declares; host-side argument validation works without a GPU (CPU only)."""
import ctypes as C
import re
from pathlib import Path

import numpy as np
import pytest

from paper_2112_00364_gb300 import smc

ROOT = Path(__file__).resolve().parent.parent


def _declared_functions():
    names = set()
    for h in sorted((ROOT / "include").glob("*.h")):
        text = h.read_text()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(smc_\w+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = smc.lib()
    names = _declared_functions()
    assert len(names) >= 10
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_version_string():
    assert "sm_103a" in smc.version()


def test_register_rejects_bad_descriptions():
    L = smc.lib()
    d = smc.ModelDesc()
    h = C.c_void_p()
    d.kind = 99
    assert L.smc_model_register(C.byref(d), C.byref(h)) == smc.EINVAL
    assert b"kind" in L.smc_last_error()
    d.kind = smc.MODEL_LG
    d.T = 0
    assert L.smc_model_register(C.byref(d), C.byref(h)) == smc.EINVAL
    assert L.smc_model_register(None, C.byref(h)) == smc.EINVAL


def test_register_rejects_bad_trees():
    import inputs

    tree = inputs.yule_tree(8, seed=1)
    bad = inputs.Tree(tree.parent.copy(), tree.left.copy(), tree.right.copy(), tree.age.copy(),
                      tree.preorder.copy())
    bad.preorder[[1, 2]] = bad.preorder[[2, 1]]  # not a left-first preorder any more
    with pytest.raises(smc.SmcError) as e:
        smc.Model("crbd", tree=bad)
    assert e.value.status == smc.EINVAL
    with pytest.raises(smc.SmcError):
        smc.Model("crbd", tree=tree, depth_cap=smc.MAX_DEPTH + 1)
    with pytest.raises(smc.SmcError):
        smc.Model("crbd", tree=tree, rho=0.0)
    with pytest.raises(smc.SmcError):
        smc.Model("rateshift", tree=tree, lam_stack_cap=0)


def test_resample_argument_checks():
    L = smc.lib()
    assert L.smc_resample(None, 10, 0.5, None, None, None, None, 0, None) == smc.EINVAL
    assert L.smc_resample_workspace_bytes(0) == 0
    assert L.smc_resample_workspace_bytes(1 << 20) > 0
    assert L.smc_gather(None, None, None, None, 10, 1, 8, None) == smc.EINVAL
    assert L.smc_sample(9, 0, 0.0, 0.0, 1, 0, 10, None, None, None) == smc.EINVAL
    # the compute-peak probe rejects bad arguments before touching a device
    assert L.smc_peak_probe(5, 10, None, None) == smc.EINVAL
    assert L.smc_peak_probe(0, 0, None, None) == smc.EINVAL


def test_particle_limit_agrees_across_header_engine_and_binding():
    header = (ROOT / "include" / "smc.h").read_text()
    m = re.search(r"#define SMC_MAX_PARTICLES \(\(\(\(int64_t\)1\) << (\d+)\) - (\d+)\)", header)
    assert m, "SMC_MAX_PARTICLES not found"
    from_header = (1 << int(m.group(1))) - int(m.group(2))
    engine = (ROOT / "paper_2112_00364_gb300" / "csrc" / "smc_engine.h").read_text()
    e = re.search(r"kMaxParticles = \(int64_t\)(0x[0-9a-f]+) - (\d+);", engine)
    assert e, "kMaxParticles not found"
    from_engine = int(e.group(1), 16) - int(e.group(2))
    assert from_header == from_engine == smc.MAX_PARTICLES
    # the last tile of a maximal run, rounded up to a whole 256-particle CTA,
    # still indexes below 2^31
    assert -(-smc.MAX_PARTICLES // 256) * 256 + 255 < 2 ** 31


def test_tile_table_rules_and_validation():
    """The tile size is a function of N from the table of N bands (host only):
    the built-in table reaches the largest run and keeps tiles in 1..256; a
    replacement table is applied and validated; None restores the built-in."""
    builtin = smc.get_tile_bands()
    assert builtin and builtin[-1][0] >= smc.MAX_PARTICLES
    for N in (1, 31, 32, 1000, 4097, 65536, 300_001, 1 << 20, smc.MAX_PARTICLES):
        t = smc.tile_size(N)
        assert 1 <= t <= min(256, N)
    assert smc.tile_size(0) == 0 and smc.tile_size(smc.MAX_PARTICLES + 1) == 0
    try:
        smc.set_tile_bands([(1000, 10, 32, 128), (smc.MAX_PARTICLES, 456, 32, 256)])
        assert smc.tile_size(900) == 90
        assert smc.tile_size(100) == 32 and smc.tile_size(5000) == 32
        assert smc.tile_size(1 << 20) == 256
        for bad in ([(1000, 0, 32, 64), (smc.MAX_PARTICLES, 1, 1, 1)],      # slots 0
                    [(smc.MAX_PARTICLES, 1, 64, 32)],                      # min > max
                    [(smc.MAX_PARTICLES, 1, 1, 512)],                      # above 256
                    [(1000, 1, 1, 1)],                                     # does not reach
                    [(1000, 1, 1, 1), (1000, 1, 1, 1)]):                   # not increasing
            with pytest.raises(smc.SmcError):
                smc.set_tile_bands(bad)
        assert smc.tile_size(900) == 90  # a rejected table leaves the current one
    finally:
        smc.set_tile_bands(None)
    assert smc.get_tile_bands() == builtin

"""The C-ABI library builds (nvcc, sm_103a), loads, and exports every entry
point that include/*.h declares; the binding declares them all too.  No
compute call is made (this runs without a GPU)."""
import ctypes
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names |= set(re.findall(r"^(?:sdm_status|const char \*)\s*(sdm_[a-z_0-9]+)\s*\(", text, re.M))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1310_1905_gb300 import build, ensemble, sdm
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_symbols()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"
    assert set(sdm.SYMBOLS) | set(ensemble.SYMBOLS) == names


def test_init_without_gpu_fails_loudly():
    import numpy as np
    import pytest
    from paper_1310_1905_gb300 import sdm
    if os.path.exists("/dev/nvidiactl"):
        pytest.skip("a GPU is present")
    with pytest.raises(sdm.SdmError) as e:
        sdm.sdm_init(dict(nx=0, ny=0, nz=0, dx=100.0, dy=100.0, dz=100.0, sd_conc=8, kernel="golovin",
                          golovin_b=1.0, init_dist="exponential", exp_mean_volume=1e-15, exp_n0=1e6),
                     np.ones(1) * 300.0, np.ones(1) * 0.01, np.ones(1))
    assert e.value.status == 3  # SDM_ECUDA: no CPU fallback

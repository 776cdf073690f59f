"""Static checks of the sweep kernel source that need no GPU: the guard band of
the ln g shadow in shared memory must cover the furthest speculative load."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KERNELS = os.path.join(ROOT, "paper_1305_5615_gb300", "csrc", "rewl_kernels.cu")

# Largest bin offset of one trial per model, from the energy change of one site:
# Ising and the 2D +-J glass dE in {-8..8} step 4 -> 2 bins; the cube dE in {-12..12}
# step 4 -> 3 bins; Potts dE in {-4..4} step 1 -> 4 bins.
MAX_TRIAL_OFFSET = {"ising": 2, "ea": 2, "ea3d": 3, "potts": 4}


def test_shadow_guard_covers_two_trial_offsets():
    """The fast loop loads trial j+1's target after a move of trial j, two offsets
    away from the current bin (which is always inside the window)."""
    src = open(KERNELS).read()
    m = re.search(r"constexpr int kGuardBins = (\d+);", src)
    assert m, "kGuardBins not found"
    assert int(m.group(1)) >= 2 * max(MAX_TRIAL_OFFSET.values())


def test_bin_offset_packing_holds_every_offset():
    """The staged form packs the offset as dbin + 8 in 8 bits and decodes it as
    (pk & 0xff) - 8; the chain forms stage it as a signed 16-bit field beside the
    trial's 16-bit index in its group (G <= 32), and the site of a trial as
    x | y << 8 | pv << 16 (x, y < 256; pv a Potts offset < 16 or a cube layer
    < 64)."""
    src = open(KERNELS).read()
    assert "(uint32_t)(ev.dbin + 8)" in src and "(int)(cur.pk & 0xffu) - 8" in src
    assert all(0 <= o + 8 <= 255 and 0 <= -o + 8 for o in MAX_TRIAL_OFFSET.values())
    assert "int16_t dbin;" in src and "uint16_t j;" in src and "mv_own.site = (uint32_t)x | ((uint32_t)y << 8) | (pv << 16);" in src
    assert "(int)(site & 0xffu), (int)((site >> 8) & 0xffu),\n" in src.replace("                                   ", "")

"""A pin set is only trusted if it fails for plausible mistakes: each of these
oracle builds carries one planted error (OR_PLANT in oracle/gldref.c, or the
``variant`` of oracle/pairnoise.py for 11, 12, 17 and 18), and at least one pin must
reject it.  The mistakes are planted on the CPU only."""
import pytest

import oracle_pins as P

PLANTS = {
    1: "K_0 not halved",
    2: "position update with a instead of b",
    3: "pair history term with the wrong sign",
    4: "inverse transform scaled by 1/m_max",
    5: "history read one step late",
    6: "a_0 = 1 in the noise target",
    7: "V_i in place of V_j in the instantaneous pair term",
    8: "conservative force with the wrong sign",
    9: "auto and cross pair correlation terms swapped",
    10: "pair-kernel table not interpolated",
    11: "pair blocks of the noise correlation matrix with the wrong sign",
    12: "pair-noise inverse transform scaled by 1/m_max",
    13: "perpendicular pair terms without the projection 1 - e e^T",
    14: "pairs closer than r_c,min dropped instead of clamped",
    15: "perpendicular factors read at the unclamped distance",
    16: "the clamped distance used for the unit vector e",
    17: "pair-noise radial factors read at the unclamped distance",
    18: "the sine part of the window's inverse transform with the wrong sign",
}


@pytest.mark.parametrize("variant", sorted(PLANTS))
def test_planted_mistake_is_caught(variant):
    caught = []
    for name, pin in P.ALL.items():
        try:
            ok, detail = pin(variant)
        except Exception as exc:  # a crash of the wrong oracle also rejects it
            ok, detail = False, repr(exc)
        if not ok:
            caught.append(name)
            break
    assert caught, f"no pin rejects plant {variant} ({PLANTS[variant]})"

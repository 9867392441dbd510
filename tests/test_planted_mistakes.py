"""The pins bite: two mistakes planted in a copy of the oracle (the E^-3 law
taken as E^-2, and a half-open coincidence window) each make the pin written
for them fail (the unchanged oracle passes those pins in the rest of the
suite).  Guards both the pins and tests/plant_mistakes.py, which runs the
full list of 56."""
import pytest

from tests import plant_mistakes as PM


@pytest.mark.parametrize("name,pin", [("e3_law", "test_material_anchors"),
                                      ("coinc_half_open_window", "test_window_edges")])
def test_planted_mistake_fails_a_pin(name, pin):
    failed = PM.run(name)
    assert any(f.startswith(pin) for f in failed), failed

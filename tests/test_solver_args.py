"""Host-side argument checks of the Python front end (no GPU needed: they run before
the library touches a device)."""
import pytest

from paper_2410_22686_gb300 import Solver


@pytest.mark.parametrize("bad", [dict(spatial="sine"), dict(precision="fp16"), dict(space="fv"),
                                 dict(smoother="zigzag"), dict(tiles="fast"), dict(tiles=3)])
def test_unknown_options_raise_value_error(bad):
    kw = dict(spatial="auto", precision="fp64", space="fd", smoother="red-black", tiles=None)
    kw.update(bad)
    with pytest.raises(ValueError):
        Solver(2, 7, 8, 1.0, 1e-3, 0.3, None, **kw)

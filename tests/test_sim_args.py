"""Host-side argument checks of the device frame simulator (they run before any device call)."""
import numpy as np
import pytest

import paper_2410_02314_gb300 as sml
from paper_2410_02314_gb300 import synth


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2410_02314_gb300 import _build

    _build.build()


class _Buf:
    """Stands in for a device buffer in calls refused before any device access."""

    def data_ptr(self):
        return 1 << 40


def _em(frame, T):
    n = len(frame)
    return synth.Emitters(frame=np.asarray(frame, np.int32), x=np.full(n, 3.0), y=np.full(n, 4.0), z=np.zeros(n),
                          photons=np.full(n, 1000.0), bg=np.full(T, 50.0))


@pytest.mark.parametrize("kw", [dict(frame=[0, 2], T=2), dict(frame=[-1], T=2), dict(frame=[0], T=2, sigma0=0.0),
                                dict(frame=[0], T=2, gain=0.0), dict(frame=[0], T=2, H=0),
                                dict(frame=[0], T=2, W=20000), dict(frame=[0], T=2, frame0=-1)])
def test_bad_simulator_arguments_are_refused(kw):
    kw = dict(kw)
    frame, T = kw.pop("frame"), kw.pop("T")
    H, W = kw.pop("H", 16), kw.pop("W", 16)
    with pytest.raises(sml.SmlError) as e:
        sml.sml_sim_frames(_em(frame, T), T, H, W, d_adu=_Buf(), **kw)
    assert e.value.code == sml.SML_ERR_BAD_ARG

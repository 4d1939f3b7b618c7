import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle

    oracle.build()
    return oracle


# Under RADTEX_CHECKED=1 the binding loads the bounds-checked build; then no
# test may leave a bounds error behind: after each test the status of every
# live context is read (and cleared) and must not be RT_ERR_OUT_OF_BOUNDS.
CHECKED = os.environ.get("RADTEX_CHECKED", "0") not in ("", "0")

if CHECKED:
    import weakref

    _contexts = weakref.WeakSet()

    def pytest_sessionstart(session):
        from paper_2301_01719_gb300 import api

        init = api.Context.__init__

        def tracked(self, *args, **kwargs):
            init(self, *args, **kwargs)
            _contexts.add(self)

        api.Context.__init__ = tracked

    @pytest.fixture(autouse=True)
    def _no_bounds_errors():
        yield
        from paper_2301_01719_gb300 import api

        for c in list(_contexts):
            if getattr(c, "handle", None) is not None and c.handle.value:
                assert api.rt_get_error(c) != api.RT_ERR_OUT_OF_BOUNDS, "a bounds check failed"

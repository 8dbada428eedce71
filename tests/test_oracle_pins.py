"""The FP64 oracle against its pins (CPU only). See tests/pins.py."""
import pytest

import oracle
import pins


@pytest.fixture(scope="module")
def o():
    return oracle.get()


@pytest.mark.parametrize("pin", pins.ALL, ids=lambda f: f.__name__)
def test_pin(o, pin):
    pin(o)

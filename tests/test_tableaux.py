"""The library-side DIRK tableaux (callers of irk.Dirk) equal the oracle's
pinned transcription of App. A entry for entry, and are lower triangular."""
import numpy as np
import pytest

from oracle import tableau
from paper_1701_07181_gb300 import tableaux


@pytest.mark.parametrize("name", ["dirk33", "esdirk65"])
def test_library_tableaux_equal_oracle(name):
    A, b, c = getattr(tableaux, name)()
    Ao, bo, co = getattr(tableau, name)()
    np.testing.assert_array_equal(A, Ao)
    np.testing.assert_array_equal(b, bo)
    np.testing.assert_array_equal(c, co)
    assert np.all(np.triu(A, 1) == 0.0)


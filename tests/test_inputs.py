"""Seeded input generators (no method arithmetic): the loop-free pattern
builders used for large request streams agree with the neighbour-list meshes."""


def test_vectorised_patterns_equal_the_mesh_builders():
    """The loop-free pattern builders (used for large request streams) give
    exactly bsr_pattern of the neighbour-list meshes."""
    import numpy as np

    from paper_1701_07181_gb300 import inputs as I
    for nx, ny in ((3, 3), (7, 5), (31, 17)):
        a, b = I.bsr_pattern(I.mesh_2d_periodic(nx, ny)), I.pattern_2d_periodic(nx, ny)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for d in ((3, 3, 3), (3, 4, 3), (5, 4, 7)):
        a, b = I.bsr_pattern(I.mesh_3d_periodic(*d)), I.pattern_3d_periodic(*d)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for T, dim in ((1000, 2), (12345, 2), (777, 3), (5000, 3)):
        a, b = I.bsr_pattern(I.mesh_for_elements(T, dim)), I.pattern_for_elements(T, dim)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])

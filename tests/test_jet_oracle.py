"""Pins of the reference jet post-processing (oracle/jet_oracle.py) on
fields whose components are known by construction."""
import numpy as np
import pytest

pytest.importorskip("scipy")
from oracle import jet_oracle as J


def field_3d():
    nz, ny, nx = 40, 20, 24
    phi = np.full((nz, ny, nx), 0.1)
    phi[0:15, 8:12, 10:14] = 0.9                 # jet column from the inlet plane: 15 x 4 x 4
    phi[20:23, 5:8, 3:6] = 0.9                   # drop of 27 cells
    phi[30:32, 14:16, 0:2] = 0.9                 # drop crossing the periodic x faces:
    phi[30:32, 14:16, 22:24] = 0.9               #   2 x 2 x 2 + 2 x 2 x 2 = 16 cells
    phi[35, 2, 2] = 0.9                          # single-cell drop
    return phi


def test_components_merge_across_periodic_faces_only():
    phi = field_3d()
    s = J.jet_stats(phi, 0.5, periodic=(False, True, True), dim=3)
    assert s["n_components"] == 4 and s["has_jet"] == 1
    assert s["breakup_length"] == 15.0
    assert s["drop_volumes"] == [1, 16, 27]
    s2 = J.jet_stats(phi, 0.5, periodic=(False, True, False), dim=3)
    assert s2["n_components"] == 5 and s2["drop_volumes"] == [1, 8, 8, 27]


def test_equivalent_diameters_and_diagonal_contacts():
    phi = np.full((10, 10), 0.1)
    phi[2, 2] = phi[3, 3] = 0.9                  # diagonal neighbours are separate (face connectivity)
    s = J.jet_stats(phi, 0.5, periodic=(False, False), dim=2)
    assert s["n_components"] == 2 and s["has_jet"] == 0
    assert np.isclose(s["mean_drop_diameter"], 2.0 * np.sqrt(1.0 / np.pi))
    phi3 = np.full((6, 6, 6), 0.1)
    phi3[2:4, 2:4, 2:4] = 0.9
    s3 = J.jet_stats(phi3, 0.5, periodic=(False, False, False), dim=3)
    assert np.isclose(s3["mean_drop_diameter"], np.cbrt(6.0 * 8 / np.pi))

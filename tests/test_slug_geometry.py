"""The slug-train measures (bubble and slug lengths, film thickness, nose) used to
compare long slug runs (Sec. 5.1) between the GPU and the oracle, pinned on colour
fields whose geometry is known by construction."""
import numpy as np
import pytest

from paper_1903_01168_gb300 import workloads as W


def _train(nx, ny, spans, rows):
    """psi = +1 (heavy) except -1 (light) on columns [a, b] (inclusive, periodic)
    of the given rows, for each (a, b) in spans."""
    psi = np.ones((ny, nx))
    for a, b in spans:
        cols = np.arange(a, b + 1) % nx
        for y in rows:
            psi[y, cols] = -1.0
    return psi


def test_lengths_film_and_crossings_of_sharp_bubbles():
    """Sharp bubbles: the centreline zero lies half way between the last light
    and the first heavy node, so a bubble of m light columns is m long; the film
    is (ny - light rows) / 2."""
    nx, ny = 200, 41
    g = W.slug_geometry(_train(nx, ny, [(50, 120)], range(10, 31)))
    assert g["n_bubbles"] == 1 and g["n_slugs"] == 1
    assert g["x_tail"] == [49.5] and g["x_nose"] == [120.5]
    assert g["bubble_len"] == 71.0 and g["slug_len"] == 129.0 and g["film"] == 10.0
    # two bubbles, one straddling x = 0 on the periodic line
    g = W.slug_geometry(_train(nx, ny, [(190, 209), (80, 99)], range(12, 29)))
    assert g["n_bubbles"] == 2 and g["n_slugs"] == 2
    assert sorted(g["x_tail"]) == [79.5, 189.5]
    assert g["bubble_len"] == 20.0 and g["slug_len"] == 80.0 and g["film"] == 12.0


def test_linear_interfaces_are_located_exactly():
    """A colour field linear across the interface puts the zero where the line
    crosses it, at fractional positions."""
    nx, ny = 64, 9
    x = np.arange(nx, dtype=np.float64)
    tail, nose = 10.3, 40.7
    pc = np.clip(np.maximum(x - nose, tail - x) / 2.0, -1.0, 1.0)   # < 0 between tail and nose
    psi = np.ones((ny, nx))
    psi[3:6] = pc
    g = W.slug_geometry(psi)
    assert g["n_bubbles"] == 1
    assert g["x_tail"][0] == pytest.approx(tail, abs=1e-12)
    assert g["x_nose"][0] == pytest.approx(nose, abs=1e-12)
    assert g["bubble_len"] == pytest.approx(nose - tail, abs=1e-12)
    assert g["slug_len"] == pytest.approx(nx - (nose - tail), abs=1e-12)


def test_open_line_counts_only_whole_bubbles():
    """On an open x axis a bubble cut by the end does not count, and a slug needs
    a bubble on both sides."""
    nx, ny = 120, 21
    psi = _train(nx, ny, [(0, 9), (30, 49), (80, 99)], range(5, 16))
    g = W.slug_geometry(psi, periodic=False)
    assert g["n_bubbles"] == 2 and g["n_slugs"] == 1
    assert g["bubble_len"] == 20.0 and g["slug_len"] == 30.0


def test_gas_column_is_the_nose_shape():
    """g(x) is the light thickness of column x: behind a round nose it grows like
    the cap's chord, 2 sqrt(r^2 - (x - x_c)^2), for a cap of radius r."""
    nx, ny, r = 128, 64, 12.0
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    yc, xc = (ny - 1) / 2.0, 60.0
    light = ((x - xc) ** 2 + (y - yc) ** 2 < r * r) | ((x < xc) & (x > 30) & (np.abs(y - yc) < r))
    psi = np.where(light, -1.0, 1.0)
    g = W.slug_geometry(psi)
    cols = np.arange(61, 71)
    chord = np.array([np.sum(np.abs(np.arange(ny) - yc) < np.sqrt(max(r * r - (c - xc) ** 2, 0.0)))
                      for c in cols])
    assert np.array_equal(g["gas"][cols], chord)

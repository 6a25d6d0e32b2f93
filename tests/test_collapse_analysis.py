"""The cold-collapse analysis (collapse.py: density centre, shell densities,
profile comparison) against closed forms, on the CPU."""
import numpy as np

from paper_1812_07313_gb300 import collapse, workloads


def test_density_centre_finds_an_offset_plummer_sphere():
    x = workloads.plummer(200000, 3) + np.array([5.0, -3.0, 2.0])
    m = np.full(len(x), 1.0 / len(x))
    c = collapse.density_centre(x, m)
    assert np.abs(c - [5.0, -3.0, 2.0]).max() < 0.03


def test_uniform_sphere_profile_is_flat_inside_and_empty_outside():
    x = workloads.uniform_sphere(400000, 4)
    m = np.full(len(x), 1.0 / len(x))
    edges, rho, count = collapse.density_profile(x, m, rmin=0.1, rmax=2.0, nbins=26)
    mid = np.sqrt(edges[1:] * edges[:-1])
    inside = (mid > 0.25) & (edges[1:] < 0.98)
    assert np.abs(rho[inside] / (3.0 / (4.0 * np.pi)) - 1.0).max() < 0.05   # M / (4/3 pi R^3)
    # a uniform sphere has no density peak: the shrinking-sphere centre wanders by ~0.02
    assert np.all(rho[edges[:-1] > 1.05] == 0.0) and count.sum() <= len(x)


def test_plummer_profile_follows_the_closed_form():
    x = workloads.plummer(400000, 5)
    m = np.full(len(x), 1.0 / len(x))
    edges, rho, count = collapse.density_profile(x, m, rmin=0.1, rmax=4.0, nbins=20)
    mid = np.sqrt(edges[1:] * edges[:-1])
    # shell average of rho(r) = 3 / (4 pi) (1 + r^2)^(-5/2): M(<r) = r^3 / (1 + r^2)^(3/2)
    menc = lambda r: r ** 3 / (1.0 + r ** 2) ** 1.5  # noqa: E731
    exact = (menc(edges[1:]) - menc(edges[:-1])) / (4.0 / 3.0 * np.pi * (edges[1:] ** 3 - edges[:-1] ** 3))
    ok = count >= 2000
    assert ok.sum() >= 10 and mid[ok].min() < 0.3
    assert np.abs(rho[ok] / exact[ok] - 1.0).max() < 0.05


def test_profile_comparison_in_dex():
    x = workloads.plummer(100000, 6)
    m = np.full(len(x), 1.0 / len(x))
    e, rho, count = collapse.density_profile(x, m)
    prof = {"r_edges": e.tolist(), "rho": rho.tolist(), "count": count.tolist()}
    doubled = dict(prof, rho=(2.0 * rho).tolist())
    res = collapse.compare_profiles([{"sim": "A", "profile": prof}, {"sim": "B", "profile": prof},
                                     {"sim": "C", "profile": doubled}])
    assert res["B_vs_A"] == 0.0
    assert abs(res["C_vs_A"] - np.log10(2.0)) < 1e-12

"""Pins of the seeded scene generators (shared inputs of oracle and GPU)."""
import numpy as np

from paper_1702_01530_gb300 import scenegen as sg


def test_splitmix64_published_vectors():
    # SplitMix64 seeded with 0: the first outputs of the reference generator
    out = sg.SplitMix64(0).u64(3).tolist()
    assert out[:2] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]
    # the counter form continues the stream across calls
    r = sg.SplitMix64(0)
    assert r.u64(1).tolist() + r.u64(2).tolist() == out


def test_uniform_and_normal_ranges():
    r = sg.SplitMix64(123)
    u = r.uniform(100000)
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01
    z = sg.SplitMix64(5).normal(100000)
    assert abs(z.mean()) < 0.02 and abs(z.std() - 1.0) < 0.02


def test_figure6_polyhedra_counts():
    # Sec. 4, Figure 6: objects of 8 vertices / 12 polygons, 12 vertices /
    # 20 polygons and 20 vertices / 36 polygons
    for f, nv, nf in ((sg.cube, 8, 12), (sg.icosahedron, 12, 20), (sg.dodecahedron, 20, 36)):
        v, faces = f()
        assert len(v) == nv and len(faces) == nf
        assert len(np.unique(faces)) == nv
        # closed surface: every edge is shared by exactly two triangles
        edges = {}
        for a, b, c in faces:
            for e in ((a, b), (b, c), (c, a)):
                k = tuple(sorted(e))
                edges[k] = edges.get(k, 0) + 1
        assert set(edges.values()) == {2}
    s = sg.config_polyhedra(5)
    assert len(s.triangles) == 2 * 12 + 2 * 20 + 36 and len(s.lights) == 1


def test_icosphere_counts_and_blob_scene_size():
    v, f = sg.icosphere(3)
    assert (len(v), len(f)) == (642, 1280)
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0)
    s = sg.config_blobs(2, n_blobs=3, n_spheres=10)
    assert len(s.triangles) == 3 * 1280 and len(s.spheres) == 10 and len(s.materials) == 13


def test_generators_are_deterministic():
    for mk in (lambda: sg.config_small(9), lambda: sg.config_blobs(4, n_blobs=5, n_spheres=30)):
        a, b = mk(), mk()
        for k in ("spheres", "triangles", "materials", "lights", "camera"):
            assert getattr(a, k).tobytes() == getattr(b, k).tobytes()
    assert sg.config_small(1).spheres.tobytes() != sg.config_small(2).spheres.tobytes()


def test_small_scene_ranges():
    s = sg.config_small(3)
    c = s.spheres["center"]
    assert (c[:, 0] >= -5).all() and (c[:, 0] <= 5).all()
    assert (c[:, 1] >= 0).all() and (c[:, 1] <= 3).all()
    assert (c[:, 2] >= -15).all() and (c[:, 2] <= -5).all()
    assert set(np.unique(s.materials["reflectivity"][:-1])) <= {0.0, 0.5}
    assert (s.W, s.H, s.max_depth, s.eye_sep, s.convergence) == (320, 240, 3, 0.065, 10.0)


def test_value_noise_hits_lattice_values_and_stays_in_range():
    ix = np.arange(-3, 4, dtype=np.float64)
    iz = np.full_like(ix, 5.0)
    v = sg.value_noise(9, ix, iz)
    k = ((ix.astype(np.int64) & 0xFFFFF) << 20) | (5 & 0xFFFFF)
    u = (sg.splitmix64_at(9, k) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
    assert np.array_equal(v, 2.0 * u - 1.0)
    x = np.linspace(-7.3, 7.9, 1001)
    w = sg.value_noise(9, x, 0.37 * x)
    assert np.abs(w).max() <= 1.0 and np.abs(np.diff(w)).max() < 0.1   # bounded and continuous


def test_splitmix64_at_matches_the_stream():
    a = sg.SplitMix64(77).u64(10)
    b = sg.splitmix64_at(77, np.arange(10))
    assert np.array_equal(a, b)


def test_terrain_counts_heights_and_cameras():
    s = sg.config_terrain(n_grid=33, n_spheres=25, W=16, H=9)
    assert len(s.triangles) == 2 * 32 * 32 and len(s.spheres) == 25 and len(s.lights) == 8
    y = s.triangles["v0"][:, 1]
    assert np.abs(y).max() <= 60.0 * (2.0 - 2.0 ** -5)          # amplitude x sum of 0.5^o
    assert (s.triangles["material"] == 0).all()
    # spheres float above the terrain surface under their centre
    c = s.spheres["center"].astype(np.float64)
    ground = 60.0 * sg.fbm(5, c[:, 0], c[:, 2], wavelength=250.0)
    assert (c[:, 1] - s.spheres["radius"] >= ground - 1e-3).all()
    cams = sg.terrain_cameras(5, 12)
    e = cams["eye"].astype(np.float64)
    assert (e[:, 1] >= 60.0 * sg.fbm(5, e[:, 0], e[:, 2], wavelength=250.0) + 20.0 - 1e-3).all()
    assert np.allclose(np.linalg.norm(cams["forward"], axis=1), 1.0, atol=1e-6)
    again = sg.config_terrain(n_grid=33, n_spheres=25, W=16, H=9)
    assert again.triangles.tobytes() == s.triangles.tobytes()

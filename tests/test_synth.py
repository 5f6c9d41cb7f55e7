"""The seeded synthetic workloads have the sizes, value ranges and structure the design states
(and the same seed gives the same arrays): box64, spiral256 and its 512^2 / 32,768-triangle form,
the 1024^2 displaced sphere, the 64-problem batch and the 256^3 volume's generator."""
import numpy as np

from paper_2309_15676_gb300 import synth


def _same(a, b):
    return all(np.array_equal(np.asarray(a.scene[k]), np.asarray(b.scene[k])) for k in ("positions", "tris")) and \
        np.array_equal(a.init_tex, b.init_tex) and np.array_equal(a.target_tex, b.target_tex)


def test_box64():
    w = synth.workload_box()
    s = w.scene
    assert (s["width"], s["height"], s["max_depth"], s["spp_prop"], s["spp_fd"]) == (64, 64, 3, 1, 1)
    assert w.init_tex.shape == (32, 32, 3) and 0.1 <= w.init_tex.min() and w.init_tex.max() <= 0.9
    assert len(s["quads"]) == 1 and np.allclose(s["quads"][0][9:], 10.0)          # the ceiling light
    assert len(s["spheres"]) == 1 and np.isclose(s["spheres"][0][3], 0.4)
    assert _same(w, synth.workload_box())


def test_spiral256_and_its_512_form():
    w = synth.workload_spiral()
    s = w.scene
    # 256 segments x 16 sides x 2 triangles, the ground quad and the light quad's two triangles
    assert len(s["tris"]) == 256 * 16 * 2 + 2 + 2
    assert (s["width"], s["height"], s["max_depth"], s["spp_prop"], s["spp_fd"]) == (256, 256, 5, 2, 1)
    for tex in (w.init_tex, w.target_tex):
        assert tex.shape == (256, 256, 5)
        lo, hi = tex.reshape(-1, 5).min(0), tex.reshape(-1, 5).max(0)
        assert np.all(lo[:3] >= 0.05) and np.all(hi[:3] <= 0.95)                   # base colour
        assert lo[3] >= 0.0 and hi[3] <= 1.0 and lo[4] >= 0.1 and hi[4] <= 0.9     # metal, roughness
    assert not np.array_equal(w.init_tex, w.target_tex)                            # seeds 11 and 12
    assert _same(w, synth.workload_spiral())
    big = synth.workload_spiral(512, 512, 512, 32, 64, 8)
    assert len(big.scene["tris"]) == 512 * 32 * 2 + 4 and big.scene["max_depth"] == 8


def test_displaced_sphere():
    w = synth.workload_sphere(tex=64)
    s = w.scene
    assert len(s["tris"]) >= 320 * 320 * 2 and (s["width"], s["max_depth"]) == (1024, 8)
    assert len(s["quads"]) == 4 and s["has_env"] == 1
    assert (s["spp_prop"], s["spp_fd"]) == (4, 4)


def test_batch_of_64_uneven_problems():
    b = synth.workload_batch()
    assert len(b) == 64
    assert {p.scene["width"] for p in b} <= {64, 128, 256, 512}
    assert {p.scene["max_depth"] for p in b} <= set(range(3, 9)) and len({p.scene["max_depth"] for p in b}) > 3
    tris = [len(p.scene["tris"]) for p in b]
    assert 1000 <= min(tris) and max(tris) <= 51000
    assert {p.init_tex.shape[0] for p in b} <= {64, 128, 256, 512} and all(p.init_tex.shape[2] == 5 for p in b)
    assert len({int(p.scene["key_id"]) for p in b}) == 64                          # independent streams


def test_volume_generator():
    w = synth.workload_volume(n=16, width=16, height=16)
    s = w.scene
    assert w.init_tex.shape == (16, 16, 16, 4) and s["n_views"] == 4 and np.isclose(s["step"], 2.0 / 16)
    assert np.all(w.init_tex[..., :3] == np.float32(0.2)) and np.all(w.init_tex[..., 3] == 1.0)
    t = w.target_tex.reshape(-1, 4)
    assert t.min() >= 0.0 and t[:, 3].max() > t[:, :3].max()                     # dense blobs
    eyes = np.asarray(s["cameras"])[:, :3]
    assert np.allclose(np.linalg.norm(eyes, axis=1), 3.2, rtol=1e-6)              # circle of radius 3.2
    assert np.allclose(eyes[:, 1], 3.2 * np.sin(0.5236), rtol=1e-6)              # 30 degrees up

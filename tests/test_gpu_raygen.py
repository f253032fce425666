"""The device secondary-ray generators against the oracle-side generator on the same hits."""
import numpy as np
import pytest

import oracle
from oracle.raygen import diffuse_rays
from paper_1811_03510_gb300 import ccs, scenegen as sg

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.mark.parametrize("mirror", [False, True])
def test_secondary_rays_match_oracle_generator(mirror):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1811_03510_gb300 import build_ext
    build_ext.build()
    torch.cuda.set_device(0)
    s = sg.make_scene(8, 0.05, 3, 1, gregory_ring=True)
    cam = sg.pinhole_rays(160, 90)
    o = oracle.intersect(s.P, s.types, cam.soa(), L=8)
    sc = ccs.Scene(s.P, s.types)
    rays = ccs.rays_to_device(cam.soa())
    hits = [torch.from_numpy(np.where(o["pid"] != 0xFFFFFFFF, o["t"], np.inf).astype(np.float32)).cuda(),
            torch.from_numpy(o["u"]).cuda(), torch.from_numpy(o["v"]).cuda(),
            torch.from_numpy(o["pid"].view(np.int32)).cuda()]
    planes = ccs.gen_mirror(sc, rays, hits) if mirror else ccs.gen_diffuse(sc, rays, hits, seed=7)
    torch.cuda.synchronize()
    got = [p.cpu().numpy() for p in planes]
    ref = diffuse_rays(s.P, s.types, cam.soa(), o, seed=7, mirror=mirror)
    act = ref[7] >= ref[6]
    assert act.sum() > 1000
    assert np.array_equal(got[7] >= got[6], act)
    for k in range(6):   # origin and direction, FP32 kernel against FP64 generator
        np.testing.assert_allclose(got[k][act], ref[k][act], atol=2e-5)
    sc.close()

"""The autotuner returns a valid configuration whose rendering matches the
default configuration's, and times every variant it chose from."""
import numpy as np
import pytest
import torch

from paper_2505_05643_gb300 import binding as B
from paper_2505_05643_gb300 import render as R
from paper_2505_05643_gb300 import synth
from paper_2505_05643_gb300 import tune

pytestmark = pytest.mark.gpu


def test_autotune_choice_renders_the_same_image():
    rng = np.random.default_rng(51)
    g = synth.scale_rot_to_tri(synth.gaussians_anisotropic(rng, 4000, ratio_max=1e3), 1e-4)
    pl = synth.planes_random(rng, [(96, 96), (64, 128), (40, 40)])
    params = torch.from_numpy(R.pack_params(g, B.UG_COV_TRI)).cuda()
    targets = torch.from_numpy(synth.target_images(rng, pl["total_pixels"])).cuda()
    cfg, table = tune.autotune(len(g["logit"]), pl, params, targets, B.UG_COV_TRI)
    assert set(table) == {16, 8}
    for tile, t in table.items():
        assert len(t["fwd"]) == B.ug_num_variants(tile)
        assert len(t["bwd"]) == B.ug_num_variants_bwd(tile)
        assert all(x > 0 for x in t["fwd"] + t["bwd"]) and t["pre_sort"] > 0
    assert cfg.tile in (8, 16) and 0 <= cfg.variant < B.ug_num_variants(cfg.tile)
    assert 0 <= cfg.variant_bwd < B.ug_num_variants_bwd(cfg.tile)
    best = min(table, key=lambda k: table[k]["total"])
    assert cfg.tile == best
    img_t, _ = R.Renderer(len(g["logit"]), pl, cfg).forward(params)
    img_d, _ = R.Renderer(len(g["logit"]), pl, R.make_config(cov_param=B.UG_COV_TRI)).forward(params)
    torch.cuda.synchronize()
    a, b = img_t.cpu().numpy(), img_d.cpu().numpy()
    assert np.allclose(a, b, rtol=1e-5, atol=1e-7)

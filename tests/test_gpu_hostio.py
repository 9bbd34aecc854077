"""HostPipeline: steps over pinned host inputs with overlapped transfers give the results of
the same steps run one after another (images bit for bit, gradients within float32
atomic-summation noise), for inputs that differ from step to step."""
import numpy as np
import pytest
import torch

import scenegen as sg
from paper_2504_17954_gb300.hostio import HostPipeline, block_views, pack_host
from paper_2504_17954_gb300.rasterizer import ATTRS
from tests import _gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("graphs", [True, False], ids=["graphs", "eager"])
def test_pipeline_matches_sequential_steps(graphs):
    base = sg.tiny_scene(3000, 64, 48, 81, log_scale_mu=-3.3, n_models=2)
    rng = np.random.default_rng(81)
    cams = [sg.look_at(3.0 * sg.random_direction(rng), 64, 48), sg.look_at(3.0 * sg.random_direction(rng), 48, 40)]
    w = sg.Workload("hostio", base.models, cams, sg.random_edits(base.models, seed=82),
                    bg=np.array([0.1, 0.2, 0.05], np.float32))
    rast, comp, table = _gpu.setup(w)
    rast.forward(comp, table)  # sizes the pair buffer
    dl = torch.randn((rast.n_pix, 4), device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    rast.backward(comp, table, dl)
    torch.cuda.synchronize()
    K = 4
    host_in = []
    for k in range(K):  # a different set of means per step
        blk = pack_host(comp)
        block_views(blk, comp.n)[0].add_(torch.from_numpy(rng.normal(0, 0.01, (comp.n, 3)).astype(np.float32)))
        host_in.append(blk)
    host_img = [torch.empty((rast.n_pix, 4), dtype=torch.float32).pin_memory() for _ in range(K)]
    host_grad = [torch.empty_like(b).pin_memory() for b in host_in]
    pipe = HostPipeline(rast, comp.model_id, comp.n_models, table, dl, graphs=graphs)
    pipe.run(host_in, host_img, host_grad)
    torch.cuda.synchronize()
    for k in range(K):
        views = block_views(host_in[k].cuda(), comp.n)
        for t, name in zip(views, ATTRS):
            getattr(comp, name).copy_(t.reshape(getattr(comp, name).shape))
        img = rast.forward(comp, table, mode="capacity").clone()
        grad, _ = rast.backward(comp, table, dl)
        torch.cuda.synchronize()
        assert torch.equal(host_img[k], img.cpu()), k
        gv = block_views(host_grad[k], comp.n)
        for t, name in zip(gv, ATTRS):
            ref = getattr(grad, name).cpu().reshape(t.shape)
            assert float((t - ref).abs().max()) <= 1e-5 * max(1.0, float(ref.abs().max())), (k, name)

"""The learned initialiser in use: trained by the library's own kernels on NNFs that
Alg. 1 computes, it must lower the training loss, let two Alg. 1 iterations reach the
energy of the plain 6-iteration search on an unseen clip, and leave the refinement
bit-exact (the oracle, given the same initial field, computes the same NNF)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

H = W = 512


@pytest.fixture(scope="module")
def trained():
    """The benchmark's recipe: 6 seeded 24-frame clips, 1200 pairs, 2500 Adam steps."""
    import torch
    import paper_2311_09265_b300 as fbp
    from paper_2311_09265_b300 import initnet_train as T
    fbp.build()
    ctx = fbp.Context(0)
    net, hist, _, _ = T.train_default(ctx, H, W, max_pairs=256)
    torch.cuda.synchronize()
    yield fbp, ctx, net, hist
    net.close()
    ctx.close()


def test_training_lowers_the_loss(trained):
    fbp, ctx, net, hist = trained
    first, last = hist[0][1], hist[-1][1]
    assert np.isfinite(last) and last < 0.5 * first
    assert net.status() == 0


def test_two_learned_iterations_reach_the_plain_search_energy(trained):
    import torch
    fbp, ctx, net, _ = trained
    g, s = synth.make_clip("blend_512_16f")          # held out: not among the training seeds
    gd, sd = torch.tensor(g, device="cuda"), torch.tensor(s, device="cuda")
    ctx.set_initnet(net)
    energies = {}
    for name, iters, flags in (("plain6", 6, fbp.FB_FLAG_REPORT_ENERGY),
                               ("plain2", 2, fbp.FB_FLAG_REPORT_ENERGY),
                               ("learned1", 1, fbp.FB_FLAG_REPORT_ENERGY | fbp.FB_FLAG_LEARNED_INIT),
                               ("learned2", 2, fbp.FB_FLAG_REPORT_ENERGY | fbp.FB_FLAG_LEARNED_INIT)):
        p = fbp.Params.make(5, iters, 1, 0, 31)
        p.flags = flags
        fbp.fb_blend_window(ctx, gd, sd, 15, p)
        e, c = ctx.energy()
        energies[name] = e / c
    ctx.set_initnet(None)
    assert energies["learned2"] <= 1.01 * energies["plain6"], energies
    assert energies["learned2"] < 0.5 * energies["plain2"], energies
    assert energies["learned1"] < energies["plain2"], energies


def test_refinement_from_the_learned_field_is_bit_exact(trained):
    import torch
    fbp, ctx, net, _ = trained
    g, _ = synth.small_clip(3, H, W, seed=synth.clip_seed(4, 901), motion="affine")
    gd = torch.tensor(g, device="cuda")
    net.forward(gd[2:3].contiguous(), gd[0:1].contiguous())
    init = net.init_nnf(1)[0].contiguous()
    p = fbp.Params.make(5, 2, 1, 0, 77, oracle.pair_tag(2, 0))
    Fg, Eg = fbp.fb_nnf(ctx, gd[2], gd[0], p, init_nnf=init)
    torch.cuda.synchronize()
    Fo, Eo = oracle.nnf(g[2], g[0], 5, 2, seed=77, pair_tag=oracle.pair_tag(2, 0),
                        init=init.cpu().numpy())
    assert (Fg.cpu().numpy() == Fo).all()
    assert (Eg.cpu().numpy().view(np.uint32) == Eo).all()


def test_learned_blend_needs_an_attached_net_of_the_right_size(trained):
    import torch
    fbp, ctx, net, _ = trained
    g = torch.zeros((3, 256, 256, 3), dtype=torch.uint8, device="cuda")
    p = fbp.Params.make(5, 1)
    p.flags = fbp.FB_FLAG_LEARNED_INIT
    with pytest.raises(fbp.FastBlendError) as e:
        fbp.fb_blend_window(ctx, g, g, 3, p)          # no net attached
    assert e.value.status == fbp.FB_ERR_ARG
    ctx.set_initnet(net)
    with pytest.raises(fbp.FastBlendError) as e:
        fbp.fb_blend_window(ctx, g, g, 3, p)          # net built for 512x512
    assert e.value.status == fbp.FB_ERR_ARG
    ctx.set_initnet(None)

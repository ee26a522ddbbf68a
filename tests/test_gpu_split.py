"""One inversion's swarm split into slices (afm_pso_init_slice /
afm_pso_best_slice / afm_pso_move_slice), as processes on several GPUs run
it, here emulated on one GPU: the slices run one after the other and the
exchange of split.invert_split (minimum key, owner's position) is done on
the host.  Nothing waits on anything across slices.  The split swarm must be
afm_invert's swarm bit for bit."""
import numpy as np
import pytest

from paper_1109_0334_gb300 import workloads as W
from common import oracle_record

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def afm():
    from paper_1109_0334_gb300 import build
    build.build()
    from paper_1109_0334_gb300 import afminv
    assert torch.cuda.is_available()
    return afminv


def _split_run(afm, prob, U, cfg, world):
    from paper_1109_0334_gb300 import split
    slices = [split.Slice(prob, U, cfg, *split.slice_of(cfg.P, r, world)) for r in range(world)]
    keys = []
    pos = None
    for it in range(cfg.iters + 1):
        kmin = min(s.evaluate(it) for s in slices)
        g = split.key_index(kmin)
        pos = next(s.position(g) for s in slices if s.owns(g)).clone()
        keys.append(kmin)
        if it < cfg.iters:
            for s in slices:
                s.move(pos, it)
    return keys, pos


@pytest.mark.parametrize("name,world", [("c1", 2), ("c1", 3), ("c2", 4)])
def test_split_swarm_equals_one_swarm(orc, afm, name, world):
    spec = W.get(name, iters=12) if name == "c1" else W.get(name, cycles=10, iters=6)
    U32, _, _ = oracle_record(orc, spec)
    U = torch.from_numpy(U32).cuda()
    prob = afm.make_problem(spec)
    cfg = afm.make_pso(spec)
    keys, pos = _split_run(afm, prob, U, cfg, world)
    # the one-swarm reference: afm_pso_step driven by afm_forward_batch
    D = len(spec["free"])
    sw = afm.pso_init(cfg, D)
    ref = []
    for it in range(cfg.iters + 1):
        _, S = afm.forward_batch(prob, sw.x, U, want_defl=False)
        afm.pso_step(cfg, sw, S, it)
        ref.append(int(sw.gbest.item()))
    assert keys == ref
    g = ref[-1] & 0xFFFFFFFF
    assert torch.equal(pos, sw.pbest_x[:, g])
    # and the fused inversion's winner
    res, hist = afm.invert(prob, U, cfg)
    torch.cuda.synchronize()
    r = afm.decode_result(res)
    assert r["winner"] == g
    np.testing.assert_array_equal(r["x"][:D], pos.double().cpu().numpy())
    S_hist = [np.uint32(k >> 32).view(np.float32) for k in keys]
    np.testing.assert_array_equal(hist.cpu().numpy(), np.array(S_hist, dtype=np.float32))


def test_slice_arguments_rejected(afm):
    spec = W.get("c1")
    cfg = afm.make_pso(spec)
    with pytest.raises(afm.AfmError) as ei:
        afm.pso_init_slice(cfg, 60, 8, 2)        # 60 + 8 > 64 particles
    assert ei.value.status == afm.ERR_INVALID_ARG
    sw = afm.pso_init_slice(cfg, 0, 32, 2)
    gb = torch.zeros(2, dtype=torch.float32, device="cuda")
    with pytest.raises(afm.AfmError):
        afm.pso_move_slice(cfg, 0, sw, gb, cfg.iters)   # the last generation has no move

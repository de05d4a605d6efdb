"""Z-slab decomposition on the CPU: the partition, the halo plan, and whole decomposed runs
whose slabs are stepped by the FP64 oracle -- in one process (LocalTransport) and as 2 and 3
gloo ranks (DistTransport) -- glued back and compared bit for bit with the single-domain
oracle run, including nz not divisible by the number of ranks."""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402
from paper_1803_01262_gb300 import inputs as I  # noqa: E402
from paper_1803_01262_gb300 import slab as S  # noqa: E402


def test_partition():
    assert S.partition(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert S.partition(8, 4) == [(0, 2), (2, 4), (4, 6), (6, 8)]
    assert S.partition(5, 1) == [(0, 5)]
    for nz in range(2, 40):
        for w in range(1, nz // 2 + 1):
            p = S.partition(nz, w)
            assert p[0][0] == 0 and p[-1][1] == nz
            assert all(a[1] == b[0] for a, b in zip(p, p[1:]))
            sizes = [b - a for a, b in p]
            assert max(sizes) - min(sizes) <= 1 and min(sizes) >= S.HALO
    with pytest.raises(ValueError):
        S.partition(5, 3)   # a slab of one plane cannot hold its neighbour's halo


def test_halo_plan_fills_every_halo_plane_from_the_right_global_plane():
    """Follow every message of every rank through global plane numbers: each halo plane of
    each slab receives the owned plane of the same global index (periodic)."""
    for nz, w in ((9, 2), (10, 3), (12, 4), (4, 2), (7, 1)):
        slabs = S.partition(nz, w)
        got = {}
        for r in range(w):
            sends, recvs = S.halo_plan(r, w, slabs)
            for m in sends:
                zb_s = slabs[m.sender][0]
                zb_r = slabs[m.receiver][0]
                for j in range(S.HALO):
                    g_src = zb_s + (m.src + j - S.HALO)
                    assert slabs[m.sender][0] <= g_src < slabs[m.sender][1]   # an owned plane
                    got[(m.receiver, m.dst + j)] = g_src % nz
                    want = (zb_r + (m.dst + j - S.HALO)) % nz
                    assert g_src % nz == want
            # receives mirror the senders' sends
            for m in recvs:
                s_sends, _ = S.halo_plan(m.sender, w, slabs)
                assert any(x.receiver == r and x.dst == m.dst and x.src == m.src and x.tag == m.tag
                           for x in s_sends)
        for r in range(w):
            own = slabs[r][1] - slabs[r][0]
            halo = [0, 1, own + 2, own + 3]
            assert sorted(k for (rr, k) in got if rr == r) == halo


def _fields(shape, seed):
    h = 1.0 / max(shape)
    phi = I.random_phi(shape, seed, smooth=True)
    u, v, w = I.random_velocity(shape, h, 8, 3, seed + 1)
    return phi, u, v, w, h


def _oracle_stepper(h, dt, eps, gamma):
    def step(p, u, v, w, vs):
        out = oracle.step(p.numpy(), u.numpy(), v.numpy(), w.numpy(), h, dt, eps, gamma, vs)
        return torch.from_numpy(out)
    return step


@pytest.mark.parametrize("shape,world", [((9, 6, 7), 1), ((9, 6, 7), 2), ((10, 5, 8), 3), ((12, 4, 6), 4)])
def test_local_slabs_equal_single_domain_oracle(shape, world):
    phi, u, v, w, h = _fields(shape, 11 + world)
    eps, gamma = 1.2 * h, 1.0
    dt = 0.1 * h * h / (gamma * eps)
    T = [torch.from_numpy(x) for x in (phi, u, v, w)]
    stepper = _oracle_stepper(h, dt, eps, gamma)
    doms = [S.SlabDomain(r, world, *T, h, stepper=stepper) for r in range(world)]
    run = S.SlabRun(doms, S.LocalTransport())
    ref = phi
    for i in range(3):
        vs = [1.0, -0.5, 0.8][i]
        run.step(dt, eps, gamma, vs)
        ref = oracle.step(ref, u, v, w, h, dt, eps, gamma, vs)
    glued = run.gather_local().numpy()
    assert np.array_equal(glued, ref)   # bit for bit
    st, rs = run.stats(), oracle.stats(ref, h ** 3, np.finfo(np.float64).eps)
    assert st["sum"] == pytest.approx(rs["sum"], rel=1e-13)
    assert st["min"] == rs["min"] and st["max"] == rs["max"]
    assert st["n_strict"] == rs["n_strict"] and st["n_tol"] == rs["n_tol"]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out, shape):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    phi, u, v, w, h = _fields(shape, 5)
    eps, gamma = 1.2 * h, 1.0
    dt = 0.1 * h * h / (gamma * eps)
    T = [torch.from_numpy(x) for x in (phi, u, v, w)]
    d = S.SlabDomain(rank, ws, *T, h, stepper=_oracle_stepper(h, dt, eps, gamma))
    run = S.SlabRun([d], S.DistTransport())
    for i in range(4):
        run.step(dt, eps, gamma, 1.0 - 0.3 * i)
    st = run.stats()
    np.save(os.path.join(out, f"slab{rank}.npy"), d.owned_view().numpy())
    with open(os.path.join(out, f"stats{rank}.json"), "w") as f:
        json.dump(dict(st, z=[d.z_begin, d.z_end]), f)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("ws,shape", [(2, (9, 6, 10)), (3, (11, 7, 5)), (3, (6, 4, 4))])
def test_gloo_ranks_equal_single_domain_oracle(tmp_path, ws, shape):
    mp.spawn(_rank_main, args=(ws, _free_port(), str(tmp_path), shape), nprocs=ws, join=True)
    phi, u, v, w, h = _fields(shape, 5)
    eps, gamma = 1.2 * h, 1.0
    dt = 0.1 * h * h / (gamma * eps)
    ref = phi
    for i in range(4):
        ref = oracle.step(ref, u, v, w, h, dt, eps, gamma, 1.0 - 0.3 * i)
    parts, stats = [], []
    for r in range(ws):
        parts.append(np.load(tmp_path / f"slab{r}.npy"))
        stats.append(json.load(open(tmp_path / f"stats{r}.json")))
    assert [s["z"] for s in stats] == [list(z) for z in S.partition(shape[0], ws)]
    assert np.array_equal(np.concatenate(parts, axis=0), ref)   # bit for bit
    rs = oracle.stats(ref, h ** 3, np.finfo(np.float64).eps)
    for st in stats:   # every rank holds the same combined statistics
        assert st["sum"] == stats[0]["sum"]
        assert st["sum"] == pytest.approx(rs["sum"], rel=1e-13)
        assert st["min"] == rs["min"] and st["max"] == rs["max"] and st["n_tol"] == rs["n_tol"]

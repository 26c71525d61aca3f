"""The multi-GPU partition (Sec. III-E, Fig. 4) on CPU ranks: two gloo processes each own half
of the lattice (whole domains, an even number per rank, so the global two-colouring holds),
run the oracle's multiplicative Schwarz sweeps on their own domains with one exchange of
boundary planes per half-sweep, and all-reduce an inner product.  The gathered result must
equal the single-process oracle's."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1412_2629_gb300 import partition as PT

DIMS, DOMAIN, GRID = (16, 4, 4, 4), (4, 2, 2, 2), (2, 1, 1, 1)
KAPPA, CSW, I_S, I_D = 0.124, 1.2, 2, 3


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    import synth
    from oracle import dd as DD
    from oracle import wilson as W
    from paper_1412_2629_gb300 import partition as P
    try:
        dist.init_process_group("gloo", rank=rank, world_size=world)
        blk = P.plan(DIMS, DOMAIN, GRID)[rank]
        x0, ex = blk.offset[0], blk.extent[0]
        U = synth.random_su3_field(DIMS, 0.5, 7).numpy()
        f = synth.gaussian_source(DIMS, 8)
        # the owned block plus one halo plane on each side in x (axis 3 of [t, z, y, x, ...])
        xs = [(x0 - 1 + i) % DIMS[0] for i in range(ex + 2)]
        U_ext = U[:, :, :, xs]
        F_ext = W.field_strength(U_ext)                 # correct on the owned planes
        own = slice(1, ex + 1)
        U_own, f_own = U_ext[:, :, :, own], f[:, :, :, x0:x0 + ex]
        F_own = {k: v[:, :, :, own] for k, v in F_ext.items()}
        solver = DD.BlockSolver(U_own, F_own, KAPPA, CSW, DD.Domains(blk.extent, DOMAIN))
        u_ext = np.zeros(U_ext.shape[:4] + (4, 3), dtype=np.complex128)
        left, right = blk.neighbours[(0, -1)], blk.neighbours[(0, +1)]

        def exchange():
            # every rank publishes its first and last owned planes; each takes its
            # neighbours' (the left neighbour's last plane, the right neighbour's first)
            mine = torch.from_numpy(np.stack([u_ext[:, :, :, 1], u_ext[:, :, :, ex]]).copy())
            mine = torch.view_as_real(mine)
            got = [torch.empty_like(mine) for _ in range(world)]
            dist.all_gather(got, mine)
            u_ext[:, :, :, 0] = torch.view_as_complex(got[left][1]).numpy()
            u_ext[:, :, :, ex + 1] = torch.view_as_complex(got[right][0]).numpy()

        for _ in range(I_S):
            for colour in (0, 1):
                exchange()
                r = f_own - W.apply_A(U_ext, u_ext, KAPPA, CSW, F_ext)[:, :, :, own]
                u_ext[:, :, :, own] += solver.solve(r, colour, I_D)
        # the outer solver's global sum: a distributed inner product
        d = torch.tensor([np.vdot(f_own, u_ext[:, :, :, own]).real], dtype=torch.float64)
        dist.all_reduce(d)
        q.put((rank, x0, u_ext[:, :, :, own].copy(), float(d[0])))
        dist.destroy_process_group()
    except Exception as e:   # report instead of leaving the other rank waiting
        q.put((rank, -1, repr(e), 0.0))


def test_plan_rejects_odd_domain_counts():
    with pytest.raises(ValueError):
        PT.plan((24, 8, 8, 8), (4, 4, 4, 4), (2, 1, 1, 1))   # 6 domains in x: 3 per rank
    with pytest.raises(ValueError):
        PT.plan((16, 8, 8, 8), (4, 4, 4, 4), (4, 1, 1, 1))   # 1 domain per rank
    blocks = PT.plan((32, 32, 32, 64), (8, 4, 4, 4), (2, 1, 1, 2))
    assert len(blocks) == 4 and blocks[3].offset == (16, 0, 0, 32) and blocks[3].extent == (16, 32, 32, 32)
    assert blocks[0].neighbours == {(0, 1): 1, (0, -1): 1, (3, 1): 2, (3, -1): 2}
    # per half-sweep: half of each boundary plane (32 x 32 x 32 sites in x, 16 x 32 x 32 in t),
    # both sides of both partitioned directions, 48 B per face site
    assert PT.halo_bytes_per_half_sweep(blocks[0]) == 2 * (32 * 32 * 32 // 2 + 16 * 32 * 32 // 2) * 48


def test_two_rank_schwarz_equals_single_process():
    import synth
    from oracle import dd as DD
    from oracle import wilson as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
    bad = [r for r in res if r[1] < 0]
    assert not bad, bad
    U = synth.random_su3_field(DIMS, 0.5, 7).numpy()
    f = synth.gaussian_source(DIMS, 8)
    ref = DD.sap(U, W.field_strength(U), f, KAPPA, CSW, DD.Domains(DIMS, DOMAIN), I_S, I_D)
    u = np.zeros_like(ref)
    for _rank, x0, part, _d in res:
        u[:, :, :, x0:x0 + part.shape[3]] = part
    assert np.abs(u - ref).max() <= 1e-13 * np.abs(ref).max()
    dots = {round(r[3], 9) for r in res}
    assert len(dots) == 1
    assert abs(res[0][3] - np.vdot(f, ref).real) <= 1e-12 * abs(np.vdot(f, ref).real)

"""z-slab decomposition on the CPU: the plane layout and partition, and the
ring halo exchange and partial-sum gather between ranks of a gloo process
group (world sizes 2 and 3). The same exchange and gather code runs
between GPUs (NCCL tensors); the packed-buffer layout used here is the one
cacl_slab_halo documents: component-major, then plane, y, x, with the
interior planes next to a side sent and the halo planes on a side
received."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from paper_2607_25444_b300 import slab as S

HALO = S.HALO


def test_partition_aligns_interiors_to_the_tile_depth():
    assert S.partition(256, 4) == [(0, 64), (64, 64), (128, 64), (192, 64)]
    assert S.partition(64, 2) == [(0, 32), (32, 32)]
    # remainder to the last slab, starts still on multiples of 32
    assert S.partition(100, 3) == [(0, 32), (32, 32), (64, 36)]
    # too few planes for whole tiles: equal shares
    assert S.partition(30, 4) == [(0, 7), (7, 7), (14, 7), (21, 9)]
    for nz, parts in ((256, 4), (100, 3), (30, 4), (7, 7)):
        ranges = S.partition(nz, parts)
        covered = [z for z0, n in ranges for z in range(z0, z0 + n)]
        assert covered == list(range(nz))


def test_local_planes_wrap_the_global_axis():
    assert S.local_planes(0, 3, 10) == [8, 9, 0, 1, 2, 3, 4]
    assert S.local_planes(7, 3, 10) == [5, 6, 7, 8, 9, 0, 1]


def _pack(arr, n, field, side):
    """The interior planes next to `side` of a local array (comp, n + 4,
    ny, nx), flattened component-major."""
    k = S.halo_planes(field)
    z = HALO if side == 0 else HALO + n - k
    return arr[:, z:z + k].reshape(-1).clone()


def _unpack(arr, n, field, side, buf):
    k = S.halo_planes(field)
    z = HALO - k if side == 0 else HALO + n
    arr[:, z:z + k] = buf.reshape(arr.shape[0], k, *arr.shape[2:])


def _worker(rank, world, port, nz, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.distributed.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ny, nx = 3, 4
        g = torch.Generator().manual_seed(7)
        comps = {S.PHI: 1, S.F: 27, S.UA: 6}
        glob = {fld: torch.rand((c, nz, ny, nx), generator=g, dtype=torch.float64)
                for fld, c in comps.items()}
        z0, n = S.partition(nz, world)[rank]
        planes = S.local_planes(z0, n, nz)
        ex = S.DistExchange()
        for fld, full in glob.items():
            local = full[:, planes].clone()
            k = S.halo_planes(fld)
            local[:, :HALO] = -1.0  # halos unknown before the exchange
            local[:, HALO + n:] = -1.0
            lo, hi = ex.sendrecv(_pack(local, n, fld, 0), _pack(local, n, fld, 1))
            _unpack(local, n, fld, 0, lo)
            _unpack(local, n, fld, 1, hi)
            want = full[:, planes]
            # every plane the exchange fills equals the global plane
            assert torch.equal(local[:, HALO - k:HALO + n + k],
                               want[:, HALO - k:HALO + n + k]), (rank, fld)
        # partial sums: rank r holds 2 nb values (uneven nb); the gather
        # lists the phi* parts of every rank in rank order, then the chi
        # parts
        nb = 3 + rank
        local = torch.tensor([1000.0 * rank + i for i in range(2 * nb)], dtype=torch.float64)
        got = ex.gather_partials(local)
        want = [1000.0 * r + i for r in range(world) for i in range(3 + r)]
        want += [1000.0 * r + 3 + r + i for r in range(world) for i in range(3 + r)]
        assert torch.equal(got, torch.tensor(want, dtype=torch.float64))
        q.put((rank, "ok"))
    except BaseException as e:  # noqa: BLE001 - reported to the parent
        q.put((rank, repr(e)))
    finally:
        torch.distributed.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,nz", [(2, 64), (3, 40)])
def test_ring_exchange_and_partial_gather_gloo(world, nz):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, nz, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    assert sorted(out) == [(r, "ok") for r in range(world)], out

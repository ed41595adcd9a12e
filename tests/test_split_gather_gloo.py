"""The gather of the frame split on the CPU (gloo, world size 2): each rank
holds output planes in which only the pixels of its own tiles (tile t belongs
to rank t mod G) are valid; bench.gather_parts must give every rank the whole
image, each pixel taken from its tile's owner."""
import os
import socket
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def owner_map(w, h, tw, th, parts):
    tiles_x = (w + tw - 1) // tw
    ys, xs = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    return ((ys // th) * tiles_x + xs // tw) % parts


def whole_image(w, h):
    """Distinct values per pixel and plane, as a render would give."""
    idx = np.arange(h * w).reshape(h, w)
    return {"iter": idx.astype(np.int32),
            "depth": (idx * 0.25).astype(np.float32),
            "normal": np.stack([idx, -idx, idx * 2], axis=-1).astype(np.float32),
            "rgba": np.stack([idx % 251, idx % 241, idx % 239, idx % 233], axis=-1).astype(np.uint8)}


def _worker(rank, world, port, w, h, tw, th, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    wsz, r, _ = bench.dist_init()
    own = owner_map(w, h, tw, th, wsz)
    full = whole_image(w, h)
    planes = {}
    for k, v in full.items():
        mine = v.copy()
        mask = own != r
        mine[mask] = 77 + r  # what a part leaves in pixels it does not own
        planes[k] = torch.from_numpy(mine)
    gathered = {k: torch.empty((wsz,) + tuple(v.shape), dtype=v.dtype) for k, v in planes.items()}
    bench.gather_parts(planes, gathered, torch.from_numpy(own.astype(np.int64)), wsz)
    ok = all(np.array_equal(planes[k].numpy(), full[k]) for k in full)
    bench.barrier(wsz)
    dist.destroy_process_group()
    q.put((r, ok))


def test_gather_parts_puts_each_pixel_from_its_owner():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    w, h, tw, th = 37, 21, 8, 8  # ragged: partial tiles on the right and bottom
    procs = [ctx.Process(target=_worker, args=(r, 2, port, w, h, tw, th, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    assert got == [(0, True), (1, True)]


def test_owner_map_matches_binding_formula():
    """The owner formula used above is the one binding.tile_parts_of_pixels
    applies to the render's tile shape (every tile owned by exactly one part,
    parts dealt round-robin in tile order)."""
    own = owner_map(37, 21, 8, 8, 3)
    tiles = [own[y, x] for y in range(0, 21, 8) for x in range(0, 37, 8)]
    assert tiles == [t % 3 for t in range(len(tiles))]

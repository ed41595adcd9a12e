"""Frame split with a gather (each process renders the tiles t with t mod G ==
rank through dqj_render_tiles, the planes are gathered and put together by tile
owner): two processes on the one GPU, gathered over gloo, must give exactly the
image of dqj_render and the same iteration and hit counts.  The two renders
are independent (no kernel waits for another process), so sharing one GPU
changes only their timing."""
import json
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2303_14827_gb300 import scenes

pytestmark = pytest.mark.gpu


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_frame_split_gather_equals_render(tmp_path):
    import split_worker
    scene_list = [scenes.default_scene(width=320, height=240),
                  dict(scenes.batch_scenes(seed=1, n=3)[2], width=300, height=200),
                  scenes.default_scene(width=197, height=131, precision=scenes.PRECISION_FP32_RECHECK),
                  scenes.default_scene(width=160, height=120, traversal=scenes.TRAVERSAL_DE),
                  scenes.full_hd_scene(3)]
    out = str(tmp_path / "split.json")
    mp.spawn(split_worker.run, args=(2, _free_port(), scene_list, out), nprocs=2, join=True)
    report = json.load(open(out))
    assert len(report) == len(scene_list)
    for i, r in enumerate(report):
        assert all(r.values()), (i, r)

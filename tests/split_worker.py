"""One rank of the frame-split test (tests/test_gpu_split.py): renders its
part of each scene's tiles with dqj_render_tiles on cuda:0, gathers every
part's planes over gloo, and on rank 0 puts them together and compares them
with dqj_render of the whole frame."""
import os


def run(rank: int, world: int, port: int, scene_list: list, result_file: str):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2303_14827_gb300 import binding

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    binding.load()
    torch.cuda.set_device(0)
    ctx = binding.dqj_create(0)
    report = []
    try:
        for s in scene_list:
            w, h = s["width"], s["height"]
            out = binding.alloc_outputs(w, h)
            for k in ("iter", "normal", "rgba"):
                out[k].fill_(7)
            out["depth"].fill_(7.0)
            stream = torch.cuda.current_stream()
            binding.dqj_render_tiles(ctx, s, binding.outputs_of(out), stream.cuda_stream, rank, world)
            stream.synchronize()
            mine = {"iter": out["iter"][:, :w].cpu(), "depth": out["depth"][:, :w].cpu(),
                    "normal": out["normal"][:, :w].cpu(), "rgba": out["rgba"][:, :w].to(torch.int32).cpu(),
                    "stats": out["stats"].cpu()}
            gathered = {}
            for k, v in mine.items():
                lst = [torch.empty_like(v) for _ in range(world)]
                dist.all_gather(lst, v.contiguous())
                gathered[k] = lst
            owner = binding.tile_parts_of_pixels(ctx, s, world)
            untouched = all(bool(np.all(mine[k].numpy()[owner != rank] == 7)) for k in ("iter", "depth", "rgba"))
            if rank == 0:
                whole = binding.alloc_outputs(w, h)
                binding.dqj_render(ctx, s, binding.outputs_of(whole), stream.cuda_stream)
                stream.synchronize()
                same = {}
                for k in ("iter", "depth", "normal", "rgba"):
                    parts = [g.numpy() for g in gathered[k]]
                    put = np.array(parts[0])
                    for r in range(1, world):
                        put[owner == r] = parts[r][owner == r]
                    ref = whole[k][:, :w].cpu()
                    ref = (ref.to(torch.int32) if k == "rgba" else ref).numpy()
                    same[k] = bool(np.array_equal(put, ref))
                st_parts = sum(g.numpy().astype(np.int64) for g in gathered["stats"])
                st_whole = whole["stats"].cpu().numpy()
                same["class_iters"] = int(st_parts[0]) == int(st_whole[0])
                same["hits"] = int(st_parts[3]) == int(st_whole[3])
                same["others_untouched_rank0"] = untouched
                report.append(same)
    finally:
        binding.dqj_destroy(ctx)
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        import json
        with open(result_file, "w") as f:
            json.dump(report, f)

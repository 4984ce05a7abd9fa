"""Worker for the two-process (gloo) test of bench.py's replica logic."""
import json
import os
import sys


def run(rank, world, port, out_dir):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import bench
    import torch.distributed as dist
    r, w, local = bench.dist_init()
    bench.barrier(w)
    # rank r "took" 10 + 5 r ms: the job time is the slowest rank's
    ms = bench.max_over_ranks(10.0 + 5.0 * r, w)
    value = bench.job_tflops(2.0e12, ms, w)
    bench.barrier(w)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"rank": r, "world": w, "local": local, "ms": ms, "value": value,
                   "backend": dist.get_backend()}, f)
    dist.destroy_process_group()

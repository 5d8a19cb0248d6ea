"""GPU: the multi-rank path through the library itself.  Two gloo ranks
(spawned processes, both on cuda:0; their kernels are independent launches
that never wait on one another) each reweight their contiguous shard of
g g -> t tbar events with librwgt, read the cross sections as (sum,
compensation) pairs and merge them with one all_gather on the host.  Each
shard's W' equals the single-process W' of the same events bit for bit (an
event's evaluation does not depend on the launch), and the merged sums equal
the exact sums of the single-process W' within 2 ulp."""
import math
import os
import socket

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

N_EVENTS = 30011


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _reweight(rwgt, ev, mom, w, pts, dev):
    stream = torch.cuda.current_stream(dev).cuda_stream
    E = mom.shape[-1]
    with rwgt.Context(0, stream) as c:
        c.set_process("gg_tt", "fp64")
        c.set_params(ev.param_vector())
        c.set_reweight_points(pts)
        c.set_tuning(0, 128)
        dm = torch.from_numpy(np.ascontiguousarray(mom)).to(dev)
        dw = torch.from_numpy(np.ascontiguousarray(w)).to(dev)
        nb = c.workspace_bytes(E)
        ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        c.load_events(dm, dw, E, ws, nb)
        wnew = torch.empty(len(pts) * E, dtype=torch.float64, device=dev)
        c.reweight_async(wnew)
        s, comp, nbad = c.get_result_pairs(len(pts))
        return wnew.cpu().numpy().reshape(len(pts), E), s, comp, nbad


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    from paper_2312_07440_gb300 import events as ev, rwgt, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dev = torch.device("cuda", 0)
    a, b = shard.shard_range(N_EVENTS, rank, world)
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], b - a, start=a)
    wnew, s, comp, nbad = _reweight(rwgt, ev, mom, w, ev.reweight_points("gg_tt_1m"), dev)
    merged = shard.allreduce_pairs(s, comp)
    np.save(os.path.join(out_dir, f"wnew{rank}.npy"), wnew)
    if rank == 0:
        np.save(os.path.join(out_dir, "merged.npy"), merged)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_on_the_library_merge_to_the_single_process_result(tmp_path):
    import torch.multiprocessing as mp

    from paper_2312_07440_gb300 import events as ev, rwgt, shard
    mp.start_processes(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, start_method="spawn")
    merged = np.load(tmp_path / "merged.npy")
    pts = ev.reweight_points("gg_tt_1m")
    mom, w = ev.generate(ev.WORKLOADS["gg_tt_1m"], N_EVENTS)
    wnew, s, comp, nbad = _reweight(rwgt, ev, mom, w, pts, torch.device("cuda", 0))
    assert nbad == 0
    for r in range(2):
        a, b = shard.shard_range(N_EVENTS, r, 2)
        assert np.array_equal(np.load(tmp_path / f"wnew{r}.npy"), wnew[:, a:b])
    for j in range(len(pts)):
        exact = math.fsum(wnew[j])
        assert abs(merged[j] - exact) <= 2 * np.spacing(exact)
    exact_orig = math.fsum(w)
    assert abs(merged[len(pts)] - exact_orig) <= 2 * np.spacing(exact_orig)

"""LDNI benchmark: one JSON line on stdout.

Workload (one GPU): the 1,310,720-triangle noisy geodesic sphere (frequency
256, r 0.35, 4-octave radial noise of amplitude 0.05) sampled into the three
1024^2 LDNIs (one-pass sampling with the learned per-tile capacity by
default, --mode exact2 for the exact two-pass form), united per axis with a
resident LDNI set of a (2,3) torus-knot tube (16,384 triangles, sampled once
before timing), and the volume of each united image (from the same Boolean
call).  One step = that whole pass over all rays of the three images;
value = 3 * 1024^2 rays / step time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain FP64 statement of the
method) on the host cores instead; multi-GPU runs are independent replicas
(weak scaling), one process per GPU under torchrun.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "LDNI rays/s & samples/s at 1024²; learned-sized 1-pass vs exact 2-pass speedup"
RES = 1024
WORKLOAD = ("noisy geodesic sphere freq 256 (655,362 verts / 1,310,720 tris, r 0.35, 4-octave radial noise 0.05)"
            " -> 3 LDNIs at 1024^2 -> union with resident (2,3) torus-knot LDNIs -> volume of the union")


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, dist=None) -> float:
    """The largest value over all ranks (each rank times its own replica;
    the job takes as long as its slowest rank).  Works with nccl (a CUDA
    tensor) and gloo (a CPU tensor)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_step: float, steps: int, max_ms: float) -> float:
    """Units per second of the whole job: every rank processes its own
    replica of the step (weak scaling), timed by the slowest rank."""
    return world * units_per_step * steps / (max_ms * 1e-3)


# Slab slots per ray of the one-pass sampler (workspace only: a tile touches
# only the slots it reserves).  Tiles reserve in whatever order their
# blocks run, and those that no longer fit are redone exactly; eight layers
# per ray leave room for every capacity the network gives the bench mesh, so
# that no tile's place depends on that order.
SLAB_LAYERS = 8


def _meshes():
    import meshgen
    return meshgen.scale_sphere(), meshgen.torus_knot(2, 3, 0.25, 0.1, 0.035, 256, 32)


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "", 1).isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------------------
# CPU oracle leg: the oracle as it stands, on every host core (one process
# per core, each running whole units of the workload on its own)
# ----------------------------------------------------------------------------
def _oracle_step(sphere, knot_ref, axes, res):
    import oracle
    o = (-0.5, -0.5, -0.5)
    rays = 0
    for a in axes:
        L = oracle.as_f32(oracle.sample(*sphere, o, 1.0, res, a, "scan"))
        U = oracle.boolean(L, knot_ref[a], "union")
        oracle.volume(U, 1.0 / res)
        rays += res * res
    return rays


def _oracle_worker(conn, res):
    """One host core: builds the workload once, then runs oracle steps on
    command ("axes", [a, ...]) -> rays, or ("for", seconds) -> (rays, steps,
    seconds of whole 3-axis steps), until ("stop",)."""
    sys.path.insert(0, ROOT)
    import oracle
    sphere, knot = _meshes()
    o = (-0.5, -0.5, -0.5)
    knot_ref = [oracle.as_f32(oracle.sample(*knot, o, 1.0, res, a, "scan")) for a in range(3)]
    conn.send("ready")
    while True:
        msg = conn.recv()
        if msg[0] == "axes":
            conn.send(_oracle_step(sphere, knot_ref, msg[1], res))
        elif msg[0] == "for":
            t0 = time.perf_counter()
            rays = steps = 0
            while True:
                rays += _oracle_step(sphere, knot_ref, (0, 1, 2), res)
                steps += 1
                if time.perf_counter() - t0 >= msg[1]:
                    break
            conn.send((rays, steps, time.perf_counter() - t0))
        else:
            conn.close()
            return


class OraclePool:
    """One spawned process per host core, each with its own copy of the
    workload (started before any GPU work: no process is forked from a
    process that holds a CUDA context)."""

    def __init__(self, workers: int, res: int):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.conns, self.procs = [], []
        for _ in range(workers):
            a, b = ctx.Pipe()
            p = ctx.Process(target=_oracle_worker, args=(b, res), daemon=True)
            p.start()
            self.conns.append(a)
            self.procs.append(p)
        for c in self.conns:
            assert c.recv() == "ready"

    def run(self, msgs):
        for c, m in zip(self.conns, msgs):
            c.send(m)
        return [c.recv() for c in self.conns[:len(msgs)]]

    def close(self):
        for c in self.conns:
            try:
                c.send(("stop",))
            except Exception:
                pass
        for p in self.procs:
            p.join(timeout=10)


def host_cpu() -> dict:
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return {"cpu_count": os.cpu_count(), "model": model}


def cpu_baseline(pool: "OraclePool", budget_s: float = 10.0) -> dict:
    """The oracle as it stands on a bounded sample of the same workload:
    whole steps (3 images at 1024^2: sampling, union, volume) repeated for
    about budget_s, first by one core alone, then by every core at once."""
    one = pool.run([("for", budget_s / 3.0)])[0]
    res = pool.run([("for", budget_s)] * len(pool.conns))
    rays = sum(r[0] for r in res)
    steps = sum(r[1] for r in res)
    wall = max(r[2] for r in res)
    cpu = host_cpu()
    return {"value": rays / wall, "unit": "rays/s", "cores": len(pool.conns), "kind": "oracle",
            "sample": f"{steps} full steps (3 axes at {RES}^2: scan-mode FP64 sampling, union, volume) on "
                      f"{len(pool.conns)} processes, one per host core, {wall:.1f} s",
            "single_core": {"value": one[0] / one[2], "unit": "rays/s", "steps": one[1], "seconds": one[2]},
            "host": cpu}


def run_reference(args):
    ws, rank, _ = _dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    cores = max(1, os.cpu_count() or 1)
    pool = OraclePool(cores, RES)
    try:
        # a step: every core runs one image (x, y, z in turn) of the workload: oracle sampling + union + volume
        msgs = lambda k: [("axes", [(k + w) % 3]) for w in range(cores)]
        for w in range(args.warmup):
            pool.run(msgs(w))
        times = []
        rays = 0
        for k in range(args.steps):
            t0 = time.perf_counter()
            rays += sum(pool.run(msgs(k)))
            times.append(time.perf_counter() - t0)
    finally:
        pool.close()
    total = sum(times)
    value = rays / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "res": RES,
                       "reference_step": f"{cores} host processes, each one image (x, y, z in turn): "
                                         "oracle sampling + union + volume"},
            "cpu_baseline": {"value": value, "unit": "rays/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} steps of {cores} images each, one process per host core",
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": "rays/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# GPU leg
# ----------------------------------------------------------------------------
def algorithmic_bytes(kid: int, nv: int, nt: int, res: int, n: list, n_knot: list, n_union: list) -> float:
    """Bytes the method must move for one launch of kernel `kid`; every
    kernel of the step covers all three images in one launch.  n, n_knot,
    n_union: samples per image of the sphere, the knot and their union."""
    N = res * res
    mesh = 12.0 * nv + 12.0 * nt
    ns, nk, nu = float(sum(n)), float(sum(n_knot)), float(sum(n_union))
    table = {
        1: mesh + 3 * 4.0 * N,                           # count: mesh read, counts written
        5: 3 * (4.0 * N + 4.0 * (N + 1)),                # scan: counts read, offsets written
        6: mesh + 3 * 4.0 * (N + 1) + 20.0 * ns,         # fill: mesh, offsets read, samples written
        8: 3 * 4.0 * (N + 1) + 40.0 * ns,                # sort: offsets, samples read + written
        # one-pass sampling: mesh read, ray counts written, (depth, tri) slab records written
        17: mesh + 3 * 4.0 * N + 8.0 * ns,
        # gather: counts and slab records read, offsets and CSR samples written
        20: 3 * 4.0 * N + 8.0 * ns + 3 * 4.0 * (N + 1) + 20.0 * ns,
        # Boolean, two-launch form: count reads rows and depths, writes counts;
        # write reads rows, counts and the kept operands' samples, writes the result
        9: 3 * (8.0 * (N + 1) + 4.0 * N) + 4.0 * (ns + nk),
        10: 3 * (8.0 * (N + 1) + 4.0 * N + 4.0 * (N + 1)) + 20.0 * (ns + nk) + 20.0 * nu,
        # Boolean, one-launch form: both operands read, result written
        13: 3 * (8.0 * (N + 1) + 4.0 * (N + 1)) + 20.0 * (ns + nk) + 20.0 * nu,
        11: 3 * 4.0 * (N + 1) + 4.0 * nu,                # volume: offsets and depths read
    }
    return table.get(kid, 0.0)


def run_e2e(ldni, dev, grid, sv, st, K, bws, vws, ws, rays_per_step, e2e_steps, net=None, margin=0.25,
            capacities=None, nbuf=2, nstreams=1, flat=True, union_capacities=None):
    """The same step through the public API (a LearnedPlan with the step's
    network, boolean_many with the union volumes), the mesh copied from pinned host
    memory and the united LDNIs plus volumes copied back, every step.

    The host never waits for the step it has just queued: the sizes and
    status words of step k are copied to pinned memory behind its kernels
    and read at step k + 1, when step k has finished; step k's results are
    then copied back on one stream while step k + 1 computes, and step
    k + 1's mesh is copied in on another while step k computes (two input
    and nbuf result buffers; the copy-back of each image on one of
    nstreams copy streams).  flat: the three result images live in one
    allocation, each with room for union_capacities[a] samples (from a
    sizing call of the same workload; default n_A + n_B, the most a union
    can have), and come back with one copy of it, unused room included.  The
    timed region runs from the first input copy to the last result copy of
    e2e_steps steps."""
    import torch
    hv = torch.from_numpy(sv).pin_memory()
    ht = torch.from_numpy(st).pin_memory()
    cap = [int(c) for c in capacities] if capacities else [3 * grid.res * grid.res // 2] * 3
    plan = ldni.LearnedPlan(len(sv), len(st), grid, cap, slab_samples=SLAB_LAYERS * 3 * grid.res * grid.res, net=net,
                            margin=margin, feature_stride=32)
    if flat:
        ucap = [int(c) for c in union_capacities] if union_capacities else [cap[a] + K[a].n for a in range(3)]
        UF = [ldni.empty_layers_flat(grid, range(3), ucap) for _ in range(nbuf)]
        U = [u for u, _ in UF]
        flat_host = [torch.empty(f.numel(), dtype=torch.uint8, pin_memory=True) for _, f in UF]
    else:
        U = [[ldni.empty_layers(grid, a, cap[a] + K[a].capacity) for a in range(3)] for _ in range(nbuf)]
    vol_dev = [torch.zeros(3, dtype=torch.float64, device=dev) for _ in range(nbuf)]
    binfo = [torch.zeros(3, 4, dtype=torch.int64, device=dev) for _ in range(nbuf)]
    vinfo = [torch.zeros(3, 4, dtype=torch.int64, device=dev) for _ in range(nbuf)]
    meta_host = [torch.empty(10, 4, dtype=torch.int64, pin_memory=True) for _ in range(nbuf)]
    host = [] if flat else [[[torch.empty(u.offsets.numel(), dtype=torch.int32, pin_memory=True)]
                             + [torch.empty(u.capacity, dtype=torch.float32, pin_memory=True) for _ in range(4)]
                             + [torch.empty(u.capacity, dtype=torch.int32, pin_memory=True)] for u in Ub] for Ub in U]
    vol_host = [torch.empty(3, dtype=torch.float64, pin_memory=True) for _ in range(nbuf)]
    copy_streams = [torch.cuda.Stream() for _ in range(nstreams)]
    ready = [torch.cuda.Event() for _ in range(nbuf)]
    copied = [[torch.cuda.Event() for _ in range(nstreams)] for _ in range(nbuf)]
    for ev in copied:
        for e in ev:
            e.record()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    d2h = [0] * nbuf

    def copy_back(j):
        """Step j's results to the host (after its sizes are known)."""
        ready[j].synchronize()
        m = meta_host[j]
        words = m[:, 3].tolist()
        st = 0
        for r in (0, 1, 2, 3, 4, 5, 9):  # status bits of the volumes, unions and sampling
            st |= int(words[r]) & 0xffffffff
        if st:
            raise RuntimeError(f"e2e step status {st:#x}")
        nbytes = 0
        if flat:
            cs = copy_streams[0]
            cs.wait_event(ready[j])
            with torch.cuda.stream(cs):
                flat_host[j].copy_(UF[j][1], non_blocking=True)
                nbytes += UF[j][1].numel()
        for a, (Ua, hb) in enumerate(() if flat else zip(U[j], host[j])):
            cs = copy_streams[a % nstreams]
            cs.wait_event(ready[j])
            with torch.cuda.stream(cs):
                n = int(m[3 + a, 0])
                for s_, h_ in zip([Ua.offsets, Ua.depth[:n], Ua.nx[:n], Ua.ny[:n], Ua.nz[:n], Ua.tri[:n]], hb):
                    h_[:s_.numel()].copy_(s_, non_blocking=True)
                    nbytes += s_.numel() * s_.element_size()
        with torch.cuda.stream(copy_streams[0]):
            vol_host[j].copy_(vol_dev[j], non_blocking=True)
            nbytes += vol_dev[j].numel() * 8
        for cs, e in zip(copy_streams, copied[j]):
            e.record(cs)
        d2h[j] = nbytes

    dvs = [torch.empty_like(hv, device=dev) for _ in range(2)]
    dts = [torch.empty_like(ht, device=dev) for _ in range(2)]
    in_stream = torch.cuda.Stream()
    in_ready = [torch.cuda.Event(), torch.cuda.Event()]
    used = [torch.cuda.Event(), torch.cuda.Event()]
    for e in used:
        e.record()

    def copy_in(k):
        """The mesh for a step into input buffer k, on its own stream."""
        with torch.cuda.stream(in_stream):
            in_stream.wait_event(used[k])  # the step that read buffer k has finished reading it
            dvs[k].copy_(hv, non_blocking=True)
            dts[k].copy_(ht, non_blocking=True)
            in_ready[k].record(in_stream)

    def compute(k, r):
        """One step's launches on the current stream: input buffer k, result buffer r."""
        plan.run(dvs[k], dts[k])
        used[k].record()
        for e in copied[r]:  # the result buffer's last copy-back is done
            torch.cuda.current_stream().wait_event(e)
        ldni.boolean_many(plan.outs, K, "union", ws=bws, outs=U[r], infos=binfo[r], sync=False, vols=vol_dev[r])
        m = meta_host[r]  # rows: volume infos, union infos, sampling status (row 9)
        m[0:3].copy_(vinfo[r], non_blocking=True)
        m[3:6].copy_(binfo[r], non_blocking=True)
        m[9:10].copy_(plan.info.view(1, 4), non_blocking=True)

    def run(nsteps):
        """nsteps whole steps: every input copied in, every result copied back."""
        copy_in(0)
        for rep in range(nsteps):
            k = rep % 2  # input buffer
            r = rep % nbuf  # result buffer
            if rep + 1 < nsteps:
                copy_in(k ^ 1)  # the next step's mesh arrives while this step computes
            torch.cuda.current_stream().wait_event(in_ready[k])
            compute(k, r)
            ready[r].record()
            if rep > 0:
                copy_back((rep - 1) % nbuf)
        copy_back((nsteps - 1) % nbuf)
        for cs in copy_streams:
            torch.cuda.current_stream().wait_stream(cs)
        torch.cuda.current_stream().wait_stream(in_stream)

    run(3)  # warm-up
    torch.cuda.synchronize()
    # timed: e2e_steps steps from the first input copy to the last result copy
    e0.record()
    h0 = time.perf_counter()
    run(e2e_steps)
    e1.record()
    torch.cuda.synchronize()
    wall = 1e3 * (time.perf_counter() - h0) / e2e_steps
    ms = e0.elapsed_time(e1) / e2e_steps
    return {"value": ws * rays_per_step / (ms * 1e-3), "unit": "rays/s",
            "h2d_bytes_per_step": int(sv.nbytes + st.nbytes), "d2h_bytes_per_step": int(max(d2h)),
            "ms_per_step": ms, "wall_ms_per_step": wall, "steps": e2e_steps,
            "api": "paper_1009_0794_gb300 LearnedPlan.run / boolean_many (with the union volumes) into empty_layers_flat "
                   "images, sizes and status read one step later; the copy-back of a step overlaps the next step",
            "result_buffers": nbuf, "copy_streams": nstreams,
            "copy_back": "one copy of the three union images' single allocation per step" if flat else
                         "one copy per array, used samples only"}


def _capacity_net(args):
    """The per-tile capacity network: loaded from --net if given, else
    trained here on 200 seeded noisy spheres at 512^2 by the library's own
    training kernels."""
    from paper_1009_0794_gb300 import capacity
    if args.net and os.path.exists(args.net):
        return capacity.CapacityNet.load(args.net), {"source": args.net}
    t0 = time.perf_counter()
    net, meta = capacity.train_default(count=200, res=512, steps=1500)
    meta["seconds"] = time.perf_counter() - t0
    meta["source"] = "trained in this run"
    return net, meta


def _capture(lib, fn, warm=3):
    """Capture fn's launches (all on torch's current stream) into a CUDA
    graph; returns (graph, library kernels per replay)."""
    import torch
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        for _ in range(warm):
            fn()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    c0 = int(lib.ldni_launch_count())
    with torch.cuda.graph(g):
        fn()
    torch.cuda.synchronize()
    return g, int(lib.ldni_launch_count()) - c0


def _learned_vs_exact(ldni, lib, plan, lplan, vt, tt, flush, reps, kmax):
    """Sampling alone, each form replayed as one CUDA graph on the same mesh
    and GPU, L2 flushed before every replay, outputs compared bit for bit:
    exact two-pass; learned one-pass; and the one-pass form without the
    network, with a fixed capacity of 2 layers per ray (overflowing tiles
    redone exactly) and of k_max layers (the deepest ray of the mesh, so
    nothing overflows, at the price of the largest slab)."""
    import torch
    res = {}
    grid = plan.grid
    N = grid.res * grid.res
    kmax += kmax & 1
    caps = [L.capacity for L in plan.outs]
    fixed2 = ldni.LearnedPlan(vt.shape[0], tt.shape[0], grid, caps, slab_samples=SLAB_LAYERS * 3 * N, net=None,
                              layers=2)
    fixedk = ldni.LearnedPlan(vt.shape[0], tt.shape[0], grid, caps, slab_samples=kmax * 3 * N, net=None,
                              layers=kmax)
    for name, p in (("exact2", plan), ("learned1", lplan), ("fixed2", fixed2), ("fixed_kmax", fixedk)):
        g, nl = _capture(lib, lambda: p.run(vt, tt))
        res[name + "_kernels"] = nl
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        res[name + "_ms"] = float(np.median(ts))
        p.finish()
        if p is not plan:
            res[name + "_overflow_tiles"] = p.overflow_tiles()
            res[name + "_identical_output"] = all(ldni.identical(a, b) for a, b in zip(plan.outs, p.outs))
    res["speedup"] = res["exact2_ms"] / res["learned1_ms"]
    res["speedup_vs_fixed2"] = res["fixed2_ms"] / res["learned1_ms"]
    res["speedup_vs_fixed_kmax"] = res["fixed_kmax_ms"] / res["learned1_ms"]
    res["kmax"] = kmax
    res["slab_slots"] = {"learned1": SLAB_LAYERS * 3 * N, "fixed2": SLAB_LAYERS * 3 * N, "fixed_kmax": kmax * 3 * N}
    res["overflow_tiles"] = lplan.overflow_tiles()
    res["tiles"] = 3 * ldni.ntiles(plan.grid.res)
    res["identical_output"] = res["learned1_identical_output"]
    return res


def _node_classify(ldni, lib, U, flush, reps):
    """Grid-node classification (Section 5.1, Step 1) of the union's three
    images: res^3 nodes, one CUDA graph replay per measurement, L2 flushed
    before each.  Bytes: the three images read, the bit volume written."""
    import torch
    res = U[0].grid.res
    out = torch.empty(res, res, (res + 31) // 32, dtype=torch.int32, device="cuda")
    sz = __import__("ctypes").c_size_t(0)
    lib.ldni_classify_nodes_workspace_size(res, __import__("ctypes").byref(sz))
    ws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")
    info = ldni.new_info()
    g, nl = _capture(lib, lambda: ldni.classify_nodes(U, out=out, ws=ws, info=info, sync=False))
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ms = float(np.median(ts))
    nbytes = 3 * 4.0 * (res * res + 1) + 4.0 * sum(L.n for L in U) + res * res * 4.0 * ((res + 31) // 32)
    return {"workload": f"{res}^3 nodes of the union's three images (2-of-3 vote)", "ms": ms,
            "nodes_per_s": res ** 3 / (ms * 1e-3), "algorithmic_bytes": nbytes, "gbs": nbytes / (ms * 1e-3) / 1e9,
            "kernels": nl}


def _contouring(ldni, lib, U, flush, reps):
    """Contouring Steps 2-3 (Section 5.1) of the union's three images: node
    signs (Step 1), active cells, edge rules, flooding and one QEF per
    cluster, one CUDA graph replay per measurement, L2 flushed before each."""
    import ctypes
    import torch
    grid = U[0].grid
    res = grid.res
    inside = ldni.classify_nodes(U)
    cells = ldni.contour_cells(U, inside=inside)  # sizes and the reference
    bound = int(min((res - 1) ** 3, 4 * sum(L.n for L in U) + 6 * (res - 1) ** 2 + 64))
    ws = torch.empty(ldni.contour_workspace_size(res, bound), dtype=torch.uint8, device="cuda")
    out = torch.empty(bound * ldni.CELL_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    info = ldni.new_info()
    arr = (ldni._CLayers * 3)(*[L.c() for L in U])
    g = grid.c()
    nodes_out = torch.empty_like(inside)
    sz = ctypes.c_size_t(0)
    lib.ldni_classify_nodes_workspace_size(res, ctypes.byref(sz))
    nws = torch.empty(sz.value, dtype=torch.uint8, device="cuda")

    def run():
        ldni.classify_nodes(U, out=nodes_out, ws=nws, info=info, sync=False)
        lib.ldni_contour_cells(arr, ctypes.byref(g), nodes_out.data_ptr(), bound, out.data_ptr(), bound,
                               info.data_ptr(), ws.data_ptr(), ws.numel(),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))

    gr, nl = _capture(lib, run)
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        gr.replay()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    m = len(cells)
    same = out[:m * ldni.CELL_DTYPE.itemsize].cpu().numpy().tobytes() == cells.tobytes()
    ms = float(np.median(ts))
    return {"workload": f"node signs and cell vertices of the union's three {res}^2 images ({(res - 1) ** 3} cells)",
            "ms": ms, "cells_with_vertices": int(m), "vertices": int(cells["nvert"].sum()),
            "cells_per_s": (res - 1) ** 3 / (ms * 1e-3), "graph_equals_eager": bool(same), "kernels": nl}


def _packed_step(ldni, lib, args, net, n_sphere, vt, tt, kv, kt, grid, flush, reps):
    """The bench step with approximate 8-bit normals (Section 3 item 1): one
    word per sample instead of three FP32 normals.  Same learned one-pass
    sampling, three-image union with the resident knot and volumes, as one
    CUDA graph; L2 flushed before each replay."""
    import torch
    res = grid.res
    K8 = ldni.sample(kv, kt, grid, "all", check_odd=True, packed=True)
    lp = ldni.LearnedPlan(vt.shape[0], tt.shape[0], grid, n_sphere, slab_samples=SLAB_LAYERS * 3 * res * res, net=net,
                          margin=args.margin, feature_stride=32, packed=True)
    bws = torch.empty(ldni.boolean_many_workspace_size(res, 3), dtype=torch.uint8, device="cuda")
    vws = torch.empty(ldni.volume_many_workspace_size(res, 3), dtype=torch.uint8, device="cuda")
    binfo = torch.zeros(3, 4, dtype=torch.int64, device="cuda")
    vinfo = torch.zeros(3, 4, dtype=torch.int64, device="cuda")
    U8 = [ldni.empty_layers(grid, a, lp.outs[a].capacity + K8[a].capacity, packed=True) for a in range(3)]
    vols = torch.zeros(3, dtype=torch.float64, device="cuda")

    def step():
        lp.run(vt, tt)
        ldni.boolean_many(lp.outs, K8, "union", outs=U8, ws=bws, infos=binfo, sync=False, vols=vols)

    g, nl = _capture(lib, step)
    ts = []
    for _ in range(reps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        g.replay()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    lp.finish()
    ok = all(ldni.info_decode(binfo[j])["status"] == 0 for j in range(3))
    ms = float(np.median(ts))
    return {"workload": f"the bench step with 8-bit normals: learned one-pass sampling at {res}^2, "
                        "three-image union, volumes", "ms": ms, "rays_per_s": 3 * res * res / (ms * 1e-3),
            "bytes_per_sample": 12, "bytes_per_sample_fp32_normals": 20, "status_ok": bool(ok), "kernels": nl}


def _offsetting(ldni, lib, U, flush, reps):
    """Offsetting by sphere unions (Section 4.2), one CUDA graph replay per
    measurement, L2 flushed before each: the flower at 128^2 by 2.5 pixels
    (the paper's offsetting examples are at 128^2, Table 4) and the union's
    three 1024^2 images by 2 pixels."""
    import ctypes
    import torch
    import meshgen
    out = {}
    fl = meshgen.flower(512, 512)
    g128 = ldni.Grid.cube((-0.5, -0.5, -0.5), 1.0, 128)
    F = ldni.sample(torch.from_numpy(fl[0]).cuda(), torch.from_numpy(fl[1]).cuda(), g128, "all")
    for name, Ls, rpix in (("flower_128_r2.5px", F, 2.5), ("union_1024_r2px", U, 2.0)):
        grid = Ls[0].grid
        r = rpix * grid.width / grid.res
        ref = ldni.offset(Ls, r)  # exact output sizes
        outs = [ldni.empty_layers(grid, a, max(L.n, 1)) for a, L in enumerate(ref)]
        n = [int(L.n) for L in Ls]
        nn = (ctypes.c_int64 * 3)(*n)
        ws = torch.empty(ldni.offset_workspace_size(n, grid.res, r, grid.width), dtype=torch.uint8, device="cuda")
        info = ldni.new_info()
        H = (ldni._CLayers * 3)(*[L.c() for L in Ls])
        arr = (ldni._CLayers * 3)(*[o.c() for o in outs])
        cg = grid.c()

        def run():
            lib.ldni_offset(H, nn, ctypes.byref(cg), ctypes.c_float(r), 0, ctypes.c_float(0.0), arr, info.data_ptr(),
                            ws.data_ptr(), ws.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))

        g, nl = _capture(lib, run)
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        for o, q in zip(outs, ref):
            o.n = q.n
        same = all(ldni.identical(o, q) for o, q in zip(outs, ref)) if info_ok(ldni, info) else False
        ms = float(np.median(ts))
        out[name] = {"workload": f"offset of {sum(n)} samples' spheres (r = {rpix} pixels) at {grid.res}^2, "
                                 "three images", "ms": ms, "rays_per_s": 3 * grid.res ** 2 / (ms * 1e-3),
                     "spheres_per_s": sum(n) / (ms * 1e-3), "samples_out": [int(q.n) for q in ref],
                     "graph_equals_eager": bool(same), "kernels": nl}
    return out


def info_ok(ldni, info):
    return ldni.info_decode(info)["status"] == 0


def merge_bytes(N: int, nA: float, nB: float, nout: float, images: int = 3) -> float:
    """Algorithmic bytes of one Boolean of `images` images: both operands'
    offsets read and the result's written (3 x 4 B per ray), every operand
    sample read and every result sample written once (20 B each)."""
    return (2 * 4.0 + 4.0) * images * (N + 1) + 20.0 * (nA + nB) + 20.0 * nout


def _flower_knot_512(ldni, timed, peak):
    """The flower (523,264 triangles) and the (2,3) knot (16,384) at 512^2:
    sampling by both exact traversals (direct and tile-binned; the tuner
    keeps the faster) and the three Booleans of the sampled images, each one
    CUDA graph replay with L2 flushed before it."""
    import torch
    import meshgen
    g = ldni.Grid.cube((-0.5, -0.5, -0.5), 1.0, 512)
    out = {"workload": "flower 512x512 (theta, phi) grid (523,264 tris) and (2,3) torus knot (16,384 tris) at "
                       "512^2, three images each; union, intersection and difference"}
    imgs = {}
    for name, (v, t) in (("flower", meshgen.flower(512, 512)),
                         ("knot", meshgen.torus_knot(2, 3, 0.25, 0.1, 0.035, 256, 32))):
        vt, tt = torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda()
        sizes = [L.n for L in ldni.sample(vt, tt, g, "all")]
        row = {"tris": len(t), "samples": int(sum(sizes))}
        for mode in ("exact2", "binned2"):
            plan = ldni.SamplePlan(len(v), len(t), g, sizes, mode=mode)
            ms, nl = timed(lambda: plan.run(vt, tt))
            plan.finish()
            row[mode + "_ms"] = ms
            row[mode + "_rays_per_s"] = 3 * 512 * 512 / (ms * 1e-3)
            imgs.setdefault(name, plan.outs)
        row["faster"] = min(("exact2", "binned2"), key=lambda m: row[m + "_ms"])
        out[name] = row
    F, K = imgs["flower"], imgs["knot"]
    ws = torch.empty(ldni.boolean_many_workspace_size(512, 3), dtype=torch.uint8, device="cuda")
    infos = torch.zeros(3, 4, dtype=torch.int64, device="cuda")
    vols = torch.zeros(3, dtype=torch.float64, device="cuda")
    for op in ("union", "inter", "diff"):
        outs = [ldni.empty_layers(g, a, F[a].capacity + K[a].capacity) for a in range(3)]
        ms, nl = timed(lambda: ldni.boolean_many(F, K, op, outs=outs, ws=ws, infos=infos, sync=False, vols=vols))
        nout = [int(x) for x in infos[:, 0].cpu().numpy()]
        ab = merge_bytes(512 * 512, sum(L.n for L in F), sum(L.n for L in K), sum(nout))
        out[op] = {"ms": ms, "samples_out": nout, "algorithmic_bytes": ab, "gbs": ab / (ms * 1e-3) / 1e9,
                   "frac_of_measured_hbm": ab / (ms * 1e-3) / 1e9 / peak, "kernels": nl}
    return out


def _scale_sphere_2048(ldni, timed, net, margin):
    """The 1,310,720-triangle sphere at 2048^2 x 3: exact two-pass and
    learned one-pass sampling, each one CUDA graph replay, output compared."""
    import torch
    import meshgen
    v, t = meshgen.scale_sphere()
    g = ldni.Grid.cube((-0.5, -0.5, -0.5), 1.0, 2048)
    vt, tt = torch.from_numpy(v).cuda(), torch.from_numpy(t).cuda()
    sizes = [L.n for L in ldni.sample(vt, tt, g, "all")]
    N = 2048 * 2048
    exact = ldni.SamplePlan(len(v), len(t), g, sizes)
    learned = ldni.LearnedPlan(len(v), len(t), g, sizes, slab_samples=SLAB_LAYERS * 3 * N, net=net, margin=margin,
                               feature_stride=32)
    ms_e, nl_e = timed(lambda: exact.run(vt, tt))
    ms_l, nl_l = timed(lambda: learned.run(vt, tt))
    exact.finish()
    learned.finish()
    same = all(ldni.identical(a, b) for a, b in zip(exact.outs, learned.outs))
    return {"workload": "noisy geodesic sphere freq 256 (1,310,720 tris) -> 3 LDNIs at 2048^2",
            "samples": int(sum(sizes)), "exact2_ms": ms_e, "learned1_ms": ms_l,
            "rays_per_s": 3 * N / (min(ms_e, ms_l) * 1e-3), "samples_per_s": sum(sizes) / (min(ms_e, ms_l) * 1e-3),
            "learned_speedup": ms_e / ms_l, "overflow_tiles": learned.overflow_tiles(), "identical_output": same,
            "kernels": {"exact2": nl_e, "learned1": nl_l}}


def _other_workloads(ldni, lib, flush, reps, net=None, margin=0.25, peak=6800.0):
    """The flower and knot at 512^2, the sphere at 2048^2, the batched
    workload (256 meshes of 1k-200k triangles at 64..512^2, one batch call),
    the 64-step union chain of a translated torus at 512^2 (three images)
    and the volume gradient, each replayed as one CUDA graph."""
    import torch
    import meshgen
    o = (-0.5, -0.5, -0.5)

    def timed(fn):
        g, nl = _capture(lib, fn)
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            g.replay()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts)), nl

    extra = {"flower_knot_512": _flower_knot_512(ldni, timed, peak),
             "scale_sphere_2048": _scale_sphere_2048(ldni, timed, net, margin)}
    batch = meshgen.batch_meshes(256, seed=7)
    plan = ldni.BatchPlan([(v, t) for v, t, _ in batch], [ldni.Grid.cube(o, 1.0, r) for _, _, r in batch])
    ms_b, nl_b = timed(plan.run)
    rays = sum(3 * r * r for _, _, r in batch)
    tris = sum(len(t) for _, t, _ in batch)
    base = meshgen.torus(R=0.1, r=0.04, nu=100, nv=100)
    meshes = [meshgen.translate(base, d) for d in meshgen.helix_offsets(64, seed=11)]
    grid = ldni.Grid.cube(o, 1.0, 512)
    cplan = ldni.BatchPlan(meshes, [grid] * 64)
    cplan.run()
    parts = cplan.finish()
    chain_run, chain_finish = ldni.union_chain_many([[parts[k][a] for k in range(64)] for a in range(3)])
    ms_c, nl_c = timed(chain_run)
    chain_out = chain_finish()
    # the adjoint of the volume (Section 2's volume, differentiated per kept crossing) on the 200,000-
    # triangle noisy icosphere at 512^2: one launch per image into one gradient buffer
    av, at = meshgen.icosphere(100, r=0.35, noise=0.03, noise_kind="octave", seed=12)
    agrid = ldni.Grid.cube(o, 1.0, 512)
    avt = torch.from_numpy(av).cuda()
    att = torch.from_numpy(at).cuda()
    AL = ldni.sample(avt, att, agrid, "all")
    grad = torch.zeros(len(av), 3, dtype=torch.float32, device="cuda")

    def adjoint():
        grad.zero_()
        for L in AL:
            ldni.volume_grad(avt, att, L, 1.0, grad_verts=grad)

    ms_a, nl_a = timed(adjoint)
    n_a = sum(L.n for L in AL)
    ab_a = sum(8.0 * L.n + 12.0 * len(at) + 24.0 * len(av) for L in AL)  # tri_id + depth, mesh, gradient
    return {**extra, "adjoint_200k_512": {"workload": f"volume gradient of the {len(at)}-triangle noisy icosphere at 512^2, "
                                             f"three images, {n_a} kept crossings", "ms": ms_a,
                                 "crossings_per_s": n_a / (ms_a * 1e-3), "algorithmic_bytes": ab_a,
                                 "gbs": ab_a / (ms_a * 1e-3) / 1e9, "kernels": nl_a},
            "batch_256": {"workload": f"256 meshes, {tris} triangles, resolutions 64..512, three images each, "
                                      "one batch call", "ms": ms_b, "rays_per_s": rays / (ms_b * 1e-3),
                          "meshes_per_s": 256 / (ms_b * 1e-3), "kernels": nl_b},
            "union_chain_64": {"workload": "64 translated 20,000-triangle tori at 512^2: 63 unions per image, "
                                           "three images, one ldni_union_chain call", "ms": ms_c,
                               "unions_per_s": 189 / (ms_c * 1e-3), "samples_out": [int(L.n) for L in chain_out],
                               "kernels": nl_c}}


def _events(n):
    """n timing events with their CUDA handles created (torch creates an
    event lazily at its first record)."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(n)]
    for e in ev:
        e.record()
    torch.cuda.synchronize()
    return ev


def run_ours(args):
    ws, rank, local = _dist_env()
    pool = None
    if not args.no_cpu_baseline and rank == 0:
        import oracle
        oracle.build()
        pool = OraclePool(max(1, os.cpu_count() or 1), RES)  # before any CUDA work in this process

    import torch
    import paper_1009_0794_gb300 as ldni
    from paper_1009_0794_gb300 import _lib

    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = _lib.load()
    (sv, st), (kv, kt) = _meshes()
    grid = ldni.Grid.cube((-0.5, -0.5, -0.5), 1.0, RES)
    vt = torch.from_numpy(sv).to(dev)
    tt = torch.from_numpy(st).to(dev)
    # resident partner LDNIs and exact capacities from one sizing call
    K = ldni.sample(kv, kt, grid, "all", check_odd=True)
    A0 = ldni.sample(vt, tt, grid, "all", check_odd=True)
    n_sphere = [L.n for L in A0]
    plan = ldni.SamplePlan(len(sv), len(st), grid, n_sphere)
    net, train_meta = _capacity_net(args)
    lplan = ldni.LearnedPlan(len(sv), len(st), grid, n_sphere, slab_samples=SLAB_LAYERS * 3 * RES * RES, net=net,
                             margin=args.margin, feature_stride=32)
    main_plan = lplan if args.mode == "learned1" else plan
    bws = torch.empty(ldni.boolean_many_workspace_size(RES, 3), dtype=torch.uint8, device=dev)
    vws = torch.empty(ldni.volume_many_workspace_size(RES, 3), dtype=torch.uint8, device=dev)
    binfo = torch.zeros(3, 4, dtype=torch.int64, device=dev)
    vinfo = torch.zeros(3, 4, dtype=torch.int64, device=dev)
    U = [ldni.empty_layers(grid, a, plan.outs[a].capacity + K[a].capacity) for a in range(3)]
    vols = torch.zeros(3, dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def step():
        main_plan.run(vt, tt)
        # the union's volumes come out of the same call (summed while its sizes are counted)
        ldni.boolean_many(main_plan.outs, K, "union", outs=U, ws=bws, infos=binfo, sync=False, vols=vols)

    import ctypes
    for w in range(max(args.warmup, 3)):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    main_plan.finish()
    # exact union sizes (one sync, outside the timed region)
    n_union = [u.n for u in ldni.boolean_many(main_plan.outs, K, "union", outs=U, ws=bws, infos=binfo, sync=True)]

    # the whole step as one CUDA graph: one launch per step
    g_step, launches_per_step = _capture(lib, step)

    # per-kernel times: a copy of the step graph with every library kernel
    # bracketed by events, replayed (synchronised) once per measured step
    cap = 64
    ev_b, ev_e = _events(cap), _events(cap)
    arr_b = (ctypes.c_void_p * cap)(*[e.cuda_event for e in ev_b])
    arr_e = (ctypes.c_void_p * cap)(*[e.cuda_event for e in ev_e])
    ids = (ctypes.c_int32 * cap)()
    _lib.check(lib.ldni_profile_set(arr_b, arr_e, ids, cap, 0), "ldni_profile_set")
    g_prof, _ = _capture(lib, step, warm=0)
    nrec = min(int(lib.ldni_profile_recorded()), cap)
    _lib.check(lib.ldni_profile_set(None, None, None, 0, 0), "ldni_profile_set")
    kid_of = [int(ids[k]) for k in range(nrec)]

    kmax = max(int(L.counts().max()) for L in A0)  # the deepest ray of the mesh
    if args.only_step:  # the step alone (profiling runs): no comparisons, next rows or other workloads
        learned, next_rows, other = {"train": train_meta}, {}, {}
    else:
        learned = _learned_vs_exact(ldni, lib, plan, lplan, vt, tt, flush, max(10, min(args.steps, 50)), kmax)
        learned["train"] = train_meta
        next_rows = {"node_classify": _node_classify(ldni, lib, U, flush, 10)}
        next_rows.update(_offsetting(ldni, lib, U, flush, 10))
        next_rows["contour_cells"] = _contouring(ldni, lib, U, flush, 10)
        next_rows["step_packed_normals"] = _packed_step(ldni, lib, args, net, n_sphere, vt, tt, kv, kt, grid, flush,
                                                        20)
    peak_hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0)) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    if not args.only_step:
        other = _other_workloads(ldni, lib, flush, 5, net=net, margin=args.margin, peak=peak_hbm)

    # timed region: K graph replays, per-step events, L2 flushed between steps
    steps = args.steps
    st_b = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    st_e = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    clocks = ClockSampler(local)
    clocks.start()
    t_settle = time.perf_counter()  # settle clocks under load before the measured steps
    while time.perf_counter() - t_settle < args.settle:
        flush.zero_()
        g_step.replay()
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        st_b[k].record()
        g_step.replay()
        st_e[k].record()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    launches = launches_per_step * steps
    step_ms = [st_b[k].elapsed_time(st_e[k]) for k in range(steps)]
    total_ms = max_over_ranks(float(sum(step_ms)), dist)
    main_plan.finish()  # raises if any step overflowed or mis-snapped

    # per-kernel averages over the same number of profiled replays
    per_kernel = {}
    for k in range(steps):
        flush.zero_()
        g_prof.replay()
        torch.cuda.synchronize()
        for r, kid in enumerate(kid_of):
            per_kernel.setdefault(kid, []).append(ev_b[r].elapsed_time(ev_e[r]))
    reps = float(steps)
    totals = {kid: sum(v) / reps for kid, v in per_kernel.items()}
    dominant = max(totals, key=totals.get)
    launches_per_call = {kid: kid_of.count(kid) for kid in totals}
    dk_ms = per_kernel[dominant]

    rays_per_step = 3 * RES * RES
    value = whole_job_rate(ws, rays_per_step, steps, total_ms)
    samples_per_s = whole_job_rate(ws, sum(n_sphere), steps, total_ms)

    # end to end through the public API from pinned host buffers
    e2e = None if args.no_e2e else run_e2e(ldni, dev, grid, sv, st, K, bws, vws, ws, rays_per_step,
                                           max(3, min(steps, 20)), net=net, margin=args.margin,
                                           capacities=n_sphere, union_capacities=n_union)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    import json as _json
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            peaks = _json.load(fh)
    except Exception:
        pass
    peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"
    dk_avg_ms = float(np.mean(dk_ms)) if dk_ms else float("nan")
    ab = algorithmic_bytes(dominant, len(sv), len(st), RES, n_sphere, [L.n for L in K], n_union)
    achieved = ab / (dk_avg_ms * 1e-3) / 1e9
    traffic = None
    ncu_note = None
    tj = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            tj = _json.load(fh)
        name = lib.ldni_kernel_name(dominant).decode()
        if name in tj and tj[name].get("source_hash") == _source_hash(tj[name].get("unit")):
            traffic = tj[name]["bytes_per_launch"]
            ncu_note = {k: tj[name][k] for k in ("alu_pipe_pct", "issue_active_pct", "dram_pct") if k in tj[name]}
            ncu_note["from"] = "profiles/traffic.json (ncu --set full of this kernel, same sources)"
    except Exception:
        traffic = None
    stages = {}
    for k in sorted(totals):
        st_ms = totals[k] / launches_per_call[k]  # per launch
        ab_k = algorithmic_bytes(k, len(sv), len(st), RES, n_sphere, [L.n for L in K], n_union)
        stages[lib.ldni_kernel_name(k).decode()] = {
            "ms_per_step": totals[k], "launches_per_step": launches_per_call[k],
            "algorithmic_bytes_per_launch": ab_k or None,
            "gbs": (ab_k / (st_ms * 1e-3) / 1e9) if ab_k else None,
            "frac_of_measured_hbm": (ab_k / (st_ms * 1e-3) / 1e9 / peak) if ab_k else None}
    # the whole merge of the step (count and write passes of three images) against its algorithmic bytes
    N = RES * RES
    merge_ms = sum(totals.get(k, 0.0) for k in (9, 10))
    mb = merge_bytes(N, sum(n_sphere), sum(L.n for L in K), sum(n_union))
    merge = {"kernels": ["bool_count", "bool_write"], "ms_per_step": merge_ms,
             "algorithmic_bytes": mb, "gbs": mb / (merge_ms * 1e-3) / 1e9 if merge_ms else None,
             "frac_of_measured_hbm": mb / (merge_ms * 1e-3) / 1e9 / peak if merge_ms else None,
             "bytes_formula": "12 B per ray and image (both operands' offsets, the result's) + 20 B per operand "
                              "sample read + 20 B per result sample written"}
    # the whole sampling call of the step (every kernel of the learned one-pass form)
    samp_ids = (14, 15, 17, 18, 4, 5, 19, 20, 25) if args.mode == "learned1" else (1, 2, 4, 5, 6, 7, 8)
    samp_ms = sum(totals.get(k, 0.0) for k in samp_ids)
    sb = 12.0 * len(sv) + 12.0 * len(st) + 3 * 4.0 * (N + 1) + 20.0 * sum(n_sphere)
    sampling = {"ms_per_step": samp_ms, "algorithmic_bytes": sb, "gbs": sb / (samp_ms * 1e-3) / 1e9 if samp_ms else None,
                "frac_of_measured_hbm": sb / (samp_ms * 1e-3) / 1e9 / peak if samp_ms else None,
                "bytes_formula": "12 B per vertex and per triangle (mesh read once) + 4 B per CSR offset + "
                                 "20 B per sample (depth, normal, triangle id)"}
    # the dominant kernel's issue bound: its warp instructions (ncu, same sources) at 4 per SM and clock
    issue = None
    try:
        name = lib.ldni_kernel_name(dominant).decode()
        rec = tj.get(name, {}) if tj else {}
        if rec.get("warp_instructions") and rec.get("source_hash") == _source_hash(rec.get("unit")) and clk.get("sm_mhz"):
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            t_issue = rec["warp_instructions"] / (sms * 4 * clk["sm_mhz"] * 1e6) * 1e3
            issue = {"warp_instructions": rec["warp_instructions"], "ms_at_full_issue": t_issue,
                     "frac": t_issue / dk_avg_ms, "sms": sms, "sm_mhz": clk["sm_mhz"]}
    except Exception:
        issue = None
    line = {
        "metric": METRIC, "value": value, "unit": "rays/s", "n_gpus": ws, "steps": steps, "warmup": args.warmup,
        "ms_per_step": total_ms / steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "res": RES, "axes": 3, "verts": len(sv), "tris": len(st),
                   "mode": args.mode, "partner": "(2,3) torus knot tube, 8,192 verts / 16,384 tris, resident LDNIs",
                   "l2": "flushed between steps (256 MiB write, outside the per-step events)",
                   "launch": "each step is one CUDA graph replay",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
        "samples_per_s": samples_per_s,
        "samples_per_step": int(sum(n_sphere)),
        "learned_speedup": learned.get("speedup"),
        "learned": learned,
        "roofline": {"bound": "hbm", "kernel": lib.ldni_kernel_name(dominant).decode(), "achieved": achieved,
                     "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": traffic,
                     "peak_source": f"{peak_src} copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                     "algorithmic_bytes_per_launch": ab, "avg_launch_ms": dk_avg_ms, "ncu": ncu_note,
                     "issue": issue},
        "merge": merge,
        "sampling_call": sampling,
        "gpu_launches": launches,
        "clocks": clk,
        "stages_ms_per_step": stages,
        "e2e": e2e,
        "next_rows": next_rows,
        "other_workloads": other,
    }
    if pool is not None:
        try:
            line["cpu_baseline"] = cpu_baseline(pool, budget_s=args.cpu_budget)
        finally:
            pool.close()
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _source_hash(unit=None) -> str:
    """The build stamp, or with `unit` (a csrc file name) the stamp of that
    translation unit and every header."""
    from paper_1009_0794_gb300 import build as b
    return b._stamp(None if unit is None else [unit])[:16]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--only-step", action="store_true",
                    help="time the step alone (no comparisons, next rows, other workloads; for profiling)")
    ap.add_argument("--settle", type=float, default=1.0, help="seconds of untimed load before the timed steps")
    ap.add_argument("--mode", default="learned1", choices=["learned1", "exact2"])
    ap.add_argument("--margin", type=float, default=0.25)
    ap.add_argument("--net", default="", help="saved capacity network (.npz); trained when absent")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()

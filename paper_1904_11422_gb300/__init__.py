"""GB300-native E-field direct imaging (MOFF / EPIC) behind a small C-ABI.

The imaging path is hand-written CUDA for sm_103a in ``libepic.so``; the
Python side (``epic``) only marshals arguments to it.  ``synth`` draws the
seeded synthetic inputs, ``autograd`` wraps the gain gradient for PyTorch and
``shard`` splits a block over processes (by channel, or by time with one sum
of the accumulators).

Quickstart (one GPU, device buffers from PyTorch)::

    import torch
    from paper_1904_11422_gb300 import epic, synth

    w = synth.station()                       # seeded LWA-station-shaped block
    plan = epic.plan_for(w)                   # FP32 path; epic.XFORMS["dft_bf16x3"] for tensor cores
    volts = torch.from_numpy(w.volts).cuda()  # [T][C][A][P] bytes, 4+4-bit complex samples
    out = torch.empty(plan.out_shape, dtype=torch.float32, device="cuda")  # [C][4][N][N]
    epic.epic_image(plan, volts, w.n_time, out, 0)  # XX, YY, Re XY, Im XY, autocorrelations removed
    epic.epic_sync(plan)
    plan.close()

Streaming from host memory: with pinned buffers, ``epic.epic_image_host_async``
enqueues a block and returns, so the next block's copy to the device overlaps
this block's imaging; ``epic.epic_sync(plan)`` waits for every enqueued block::

    h_in = [torch.from_numpy(b).pin_memory() for b in blocks]
    h_out = [torch.empty(plan.out_shape, dtype=torch.float32).pin_memory() for _ in blocks]
    for v, o in zip(h_in, h_out):
        epic.epic_image_host_async(plan, v, w.n_time, o, 0)
    epic.epic_sync(plan)
"""
__all__ = ["epic", "synth"]

"""GB300-native E-field direct imaging (MOFF / EPIC) behind a small C-ABI.

The imaging path is hand-written CUDA for sm_103a in ``libepic.so``; the
Python side (``epic``) only marshals arguments to it.  ``synth`` draws the
seeded synthetic inputs, ``autograd`` wraps the gain gradient for PyTorch and
``shard`` splits a band of channels over processes.

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
"""
__all__ = ["epic", "synth"]

"""CUDA-event timing on an instance's own stream (torch supplies the events)."""
from __future__ import annotations

import numpy as np

from . import mprk as M


def time_steps(h: int, stream_ptr: int, steps: int) -> float:
    """Milliseconds for `steps` slow steps, events recorded on the stream the
    step graph is launched on."""
    import torch
    ext = torch.cuda.ExternalStream(stream_ptr)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(ext):
        e0.record(ext)
        M.mprk_step(h, steps)
        e1.record(ext)
    e1.synchronize()
    return float(e0.elapsed_time(e1))


def time_region(stream_ptr: int, fn) -> float:
    """Milliseconds of the work fn() enqueues on the stream (CUDA events)."""
    import torch
    ext = torch.cuda.ExternalStream(stream_ptr)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    with torch.cuda.stream(ext):
        e0.record(ext)
        fn()
        e1.record(ext)
    e1.synchronize()
    return float(e0.elapsed_time(e1))


def stage_kernel_times(h: int, stream_ptr: int, reps: int = 3):
    """(ms, cell-stages, share): the summed duration of the stage-kernel
    launches of one slow step, the cell-stages they computed, and their
    share of the step's launches, medians over `reps` slow steps run as a
    graph with an event node after every launch. The event nodes add a gap
    before each launch, so the durations run a little long; their share
    scaled by the plain graph's step time bounds the kernel's own time
    (see kernel_ms_per_step)."""
    tot, share, cells = [], [], None
    for _ in range(reps):
        ms, c = M.mprk_profile_step(h)
        stage = c > 0
        tot.append(float(ms[stage].sum()))
        share.append(float(ms[stage].sum() / ms.sum()))
        cells = int(c[stage].sum())
    return float(np.median(tot)), cells, float(np.median(share))


def kernel_ms_per_step(step_ms: float, share: float) -> float:
    """The stage kernel's time per slow step inside the step graph: its share
    of the launches (event-timed) times the plain graph's step time. It
    counts the gaps between launches to the kernels in proportion, so it is
    an upper bound of their busy time, and never exceeds the step."""
    return step_ms * share

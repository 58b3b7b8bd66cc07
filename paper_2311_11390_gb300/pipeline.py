"""Host <-> device pipelining of consecutive steps.

A step reads inputs that arrive from pinned host memory and produces results that go back to
it.  Run back to back on one stream, every step waits for its own copies.  `DoubleBuffered`
keeps two slots of per-step device buffers and three streams: step k's inputs are copied in on
the upload stream while step k-1 computes, and step k's results are copied out on the download
stream while step k+1 computes.  Events order the reuse of a slot: an upload into a slot waits
until the step that last read it has finished computing, and a compute waits until the download
of the results it will overwrite has finished.

Everything a step computes runs on the compute stream in order, so buffers outside the slots
(intermediates such as the current I or the checkpoints) are shared safely between steps.
"""
from __future__ import annotations

from typing import Callable

import torch


class DoubleBuffered:
    """Overlap host copies with compute across consecutive steps.

    make_slot() -> dict of device tensors for one step in flight (inputs and results);
    load(k, slot) enqueues step k's host -> device copies (on the current stream);
    compute(k, slot) enqueues step k's kernels; store(k, slot) enqueues its device -> host
    copies.  All three are called with torch's current stream set to the stream they run on.
    """

    def __init__(self, device: torch.device, make_slot: Callable[[], dict]):
        self.device = torch.device(device)
        self.slots = [make_slot(), make_slot()]
        self.up = torch.cuda.Stream(self.device)
        self.down = torch.cuda.Stream(self.device)

    def run(self, n: int, load, compute, store, stream: torch.cuda.Stream | None = None) -> None:
        """Enqueue n steps; returns once they are enqueued.  The given (or current) stream
        waits for the last download, so an event recorded on it afterwards closes the run."""
        main = stream if stream is not None else torch.cuda.current_stream(self.device)
        start = torch.cuda.Event()
        start.record(main)
        read_done = [None, None]   # compute of the step that last read the slot's inputs
        stored = [None, None]      # download of the slot's last results
        for k in range(n):
            s = k & 1
            slot = self.slots[s]
            loaded = torch.cuda.Event()
            with torch.cuda.stream(self.up):
                self.up.wait_event(start)
                if read_done[s] is not None:
                    self.up.wait_event(read_done[s])
                load(k, slot)
                loaded.record(self.up)
            done = torch.cuda.Event()
            with torch.cuda.stream(main):
                main.wait_event(loaded)
                if stored[s] is not None:
                    main.wait_event(stored[s])
                compute(k, slot)
                done.record(main)
            read_done[s] = done
            fin = torch.cuda.Event()
            with torch.cuda.stream(self.down):
                self.down.wait_event(done)
                store(k, slot)
                fin.record(self.down)
            stored[s] = fin
        for ev in stored:
            if ev is not None:
                main.wait_event(ev)

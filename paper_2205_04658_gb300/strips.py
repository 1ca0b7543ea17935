"""One lattice decomposed into horizontal strips of whole rows.

The update reads, at each cell, only that cell and its eight neighbours: the collision is
local, and the streaming pull moves populations by at most one cell (dt/a <= 1; Sec.
"The Standard/Classical LBM", Sec. "Boltzmann to Lattice Boltzmann").  A strip of rows
therefore steps exactly as the same rows of the whole lattice if, before every step, its
two ghost rows hold the boundary rows of the strips below and above it -- the populations
that cross each face.  The library's strip contexts (rlbm_config.strip_y0 /
strip_ny_total) keep the stirring phases and the rounding of 16-bit stores on the
lattice's own rows, and rlbm_halo_pack / rlbm_halo_unpack move one face's crossing planes
(6 of 17 padded rows for the paper's set).

  * StripSet: every strip of one lattice on the current device, exchanged by device copies
    between steps (one stream, so no kernel ever waits on another).
  * exchange(): one halo exchange between processes that each hold one strip, over
    torch.distributed point-to-point messages (gloo between host processes; the same calls
    carry device tensors between GPUs).
  * DistributedStrip: this process's strip of a lattice spread over the ranks of a process
    group, exchanged with exchange() after every step (messages staged through pinned host
    memory when the backend moves host tensors only, as gloo does).

Conserved totals of the whole lattice are the sums of the strips' totals (FP64)."""
import numpy as np

from . import rlbm


def strip_rows(ny, nstrips):
    """Row ranges [(y0, y1), ...] of nstrips near-equal strips of ny rows."""
    cuts = [ny * i // nstrips for i in range(nstrips + 1)]
    return [(cuts[i], cuts[i + 1]) for i in range(nstrips)]


def neighbours(index, count, periodic):
    """(below, above): the strips next to strip `index` of `count`, None beyond a wall."""
    below = index - 1 if index > 0 else (count - 1 if periodic else None)
    above = index + 1 if index < count - 1 else (0 if periodic else None)
    return below, above


def exchange(dist, send_lo, send_hi, recv_lo, recv_hi, rank, world, periodic, group=None):
    """One halo exchange of the strip held by `rank` (strips in rank order, bottom first):
    send_lo (this strip's face-0 message) goes to the strip below, whose recv_hi takes it;
    send_hi goes to the strip above, whose recv_lo takes it.  Faces at a wall are None.

    Messages to one peer are posted in an order that pairs them under both backends (NCCL
    pairs point-to-point messages between two ranks in the order they are posted, gloo by
    tag as well): every rank first sends down and receives from above (tag 0), then sends up
    and receives from below (tag 1).  With world = 1 the strip is its own neighbour."""
    lo, hi = neighbours(rank, world, periodic)
    if world == 1:
        if hi is not None:
            recv_hi.copy_(send_lo)
        if lo is not None:
            recv_lo.copy_(send_hi)
        return
    ops = []
    if lo is not None:
        ops.append(dist.P2POp(dist.isend, send_lo, lo, group, 0))
    if hi is not None:
        ops.append(dist.P2POp(dist.irecv, recv_hi, hi, group, 0))
    if hi is not None:
        ops.append(dist.P2POp(dist.isend, send_hi, hi, group, 1))
    if lo is not None:
        ops.append(dist.P2POp(dist.irecv, recv_lo, lo, group, 1))
    if ops:
        for w in dist.batch_isend_irecv(ops):
            w.wait()


def _strip_kwargs(nx, ny, y0, y1, kw):
    """Keyword arguments of rlbm.Lattice for the strip of rows [y0, y1) of the lattice that the
    lattice-wide keyword arguments kw describe (their arrays cut to the strip's rows)."""
    skw = {k: v for k, v in kw.items() if k not in ("solid", "init_eps", "init_ux", "init_uy")}
    skw.update(strip_y0=y0, strip_ny_total=ny)
    for k in ("init_eps", "init_ux", "init_uy"):
        if kw.get(k) is not None:
            skw[k] = np.asarray(kw[k], np.float64).reshape(ny, nx)[y0:y1]
    if kw.get("solid") is not None:
        m = np.asarray(kw["solid"], np.uint8).reshape(ny, nx)
        skw["solid"] = m[y0:y1]
        skw["strip_solid_halo"] = np.stack([m[(y0 - 1) % ny], m[y1 % ny]])
    return skw


class DistributedStrip:
    """The strip of an nx x ny lattice that this rank of a torch.distributed process group
    holds (strips in rank order, bottom first), on the current device.  Takes the keyword
    arguments of rlbm.Lattice for the whole lattice.  step(n) advances it and exchanges the
    halos with the neighbouring ranks after each step; every rank calls it together.
    device_messages: send device tensors (NCCL); False stages the messages through pinned
    host memory (gloo); None picks by the group's backend."""

    def __init__(self, dist, nx, ny, stream=None, group=None, device_messages=None, **kw):
        import torch
        self.dist, self.group = dist, group
        self.rank, self.world = dist.get_rank(group), dist.get_world_size(group)
        self.nx, self.ny = nx, ny
        self.periodic = not kw.get("walls_y", 0)
        self.y0, self.y1 = strip_rows(ny, self.world)[self.rank]
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.lat = rlbm.Lattice(nx, self.y1 - self.y0, stream=self.stream, **_strip_kwargs(nx, ny, self.y0, self.y1, kw))
        if device_messages is None:
            device_messages = dist.get_backend(group) == "nccl"
        self.device_messages = device_messages
        n = rlbm.rlbm_halo_bytes(self.lat.ctx)
        self.dev = [torch.empty(n, dtype=torch.uint8, device="cuda") for _ in range(4)]  # send lo, hi; recv lo, hi
        self.host = None if device_messages else [torch.empty(n, dtype=torch.uint8).pin_memory() for _ in range(4)]
        self.exchange()

    def exchange(self):
        import torch
        below, above = neighbours(self.rank, self.world, self.periodic)
        ctx = self.lat.ctx
        if below is not None:
            rlbm.rlbm_halo_pack(ctx, 0, self.dev[0].data_ptr())
        if above is not None:
            rlbm.rlbm_halo_pack(ctx, 1, self.dev[1].data_ptr())
        self.stream.synchronize()  # the messages are complete before another stream or the host reads them
        if self.device_messages:
            msg = self.dev
        else:
            for i in (0, 1):
                self.host[i].copy_(self.dev[i])
            msg = self.host
        exchange(self.dist, msg[0], msg[1], msg[2], msg[3], self.rank, self.world, self.periodic, self.group)
        if self.device_messages:  # the received messages are complete on torch's current stream
            self.stream.wait_stream(torch.cuda.current_stream())
        else:
            for i in (2, 3):
                self.dev[i].copy_(self.host[i])
            torch.cuda.synchronize()
        if below is not None:
            rlbm.rlbm_halo_unpack(ctx, 0, self.dev[2].data_ptr())
        if above is not None:
            rlbm.rlbm_halo_unpack(ctx, 1, self.dev[3].data_ptr())

    def step(self, n=1):
        for _ in range(n):
            self.lat.step(1)
            self.exchange()

    def moments(self):
        """This strip's eps, u^x, u^y and the lattice's totals (an FP64 sum over the ranks)."""
        import torch
        E, UX, UY, tot = self.lat.moments()
        t = torch.from_numpy(np.array(tot, dtype=np.float64))
        if self.device_messages:
            t = t.cuda()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)
        return E, UX, UY, t.cpu().numpy()

    def close(self):
        self.lat.close()


class StripSet:
    """A lattice of nx x ny cells held as `nstrips` strip contexts on the current device.
    Takes the keyword arguments of rlbm.Lattice; the lattice-wide arrays (solid, init_*)
    are cut into the strips' rows.  step(n) advances every strip and exchanges the halos
    after each step, so the ghost rows always belong to the current state."""

    def __init__(self, nx, ny, nstrips, stream=None, **kw):
        import torch
        self.nx, self.ny = nx, ny
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.periodic = not kw.get("walls_y", 0)
        self.rows = strip_rows(ny, nstrips)
        self.strips = [rlbm.Lattice(nx, y1 - y0, stream=self.stream, **_strip_kwargs(nx, ny, y0, y1, kw))
                       for (y0, y1) in self.rows]
        nbytes = rlbm.rlbm_halo_bytes(self.strips[0].ctx)
        # message buffers: [strip][face] (torch device allocations are 256-byte aligned)
        self.msg = [[torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(2)]
                    for _ in self.strips]
        self.exchange()

    def _has_face(self, i, face):
        below, above = neighbours(i, len(self.strips), self.periodic)
        return (below if face == 0 else above) is not None

    def exchange(self):
        """Pack every strip's boundary rows, then unpack each into its neighbours' ghost rows
        (all on the strips' stream)."""
        n = len(self.strips)
        for i, s in enumerate(self.strips):
            for face in (0, 1):
                if self._has_face(i, face):
                    rlbm.rlbm_halo_pack(s.ctx, face, self.msg[i][face].data_ptr())
        for i, s in enumerate(self.strips):
            below, above = neighbours(i, n, self.periodic)
            if below is not None:
                rlbm.rlbm_halo_unpack(s.ctx, 0, self.msg[below][1].data_ptr())
            if above is not None:
                rlbm.rlbm_halo_unpack(s.ctx, 1, self.msg[above][0].data_ptr())

    def step(self, n=1):
        for _ in range(n):
            for s in self.strips:
                s.step(1)
            self.exchange()

    @property
    def current_step(self):
        return self.strips[0].current_step

    def moments(self):
        """eps, u^x, u^y (ny x nx) of the whole lattice and its totals (sums of the strips')."""
        parts = [s.moments() for s in self.strips]
        E, UX, UY = (np.concatenate([p[k] for p in parts], axis=0) for k in range(3))
        return E, UX, UY, np.sum([p[3] for p in parts], axis=0)

    def get_state(self):
        parts = [s.get_state() for s in self.strips]
        return np.concatenate([p[0] for p in parts], axis=1), parts[0][1]

    def set_launch(self, ctas, stages=0, stir_rows=0):
        for s in self.strips:
            s.set_launch(ctas, stages, stir_rows)

    def close(self):
        for s in self.strips:
            s.close()
        self.strips = []

"""Domain decomposition of the lattice into slabs of time slices.

The paper runs on one node and leaves distributed memory to future work
(Sec. 1); App. A notes that the spin projection halves what a Wilson halo
must carry.  Here rank r of R owns the time slices [t0, t1) of an
N_x x N_y x N_z x N_t lattice and holds them in a slab operator of t extent
t1 - t0 + 2: slices 0 and t1 - t0 + 1 are ghost copies of the neighbouring
slabs' edge slices.  Every stencil (D_W, D_B, D_S and their daggers) reaches
one slice in t, so one ghost slice per side is the whole halo.  An apply is

    pack the two owned edge slices   (dirac_halo_pack; half spinors for D_W)
    exchange them with the neighbours (torch.distributed, or in-process)
    unpack into the ghost slices      (dirac_halo_unpack)
    D on the owned slices             (dirac_apply_range)

All vector arithmetic runs in libdirac kernels; this module marshals
tensors, moves the packed slices and, in the distributed CG, forms the N_v
step lengths on the host from the reduced dot products (as the library's own
CG does).  The global boundary phase in t is folded into the
slab's links here (the slab operator itself is created periodic in t); the
spatial phases stay with the operator (spatial extents are global).
"""
import numpy as np
import torch

from . import dirac as D


def slab_bounds(nt, world, rank):
    """Owned time slices [t0, t1) of rank `rank` among `world` slabs."""
    if not (0 <= rank < world) or world > nt:
        raise ValueError("need 0 <= rank < world <= N_t")
    return rank * nt // world, (rank + 1) * nt // world


def slab_links(U, bc, world, rank):
    """The slab's links (numpy, (t1 - t0 + 2, Nz, Ny, Nx, 4, Nc, Nc)): global
    slices t0 - 1 .. t1 (periodically), with the global boundary phase bc[3]
    folded into U_t on the global slice N_t - 1."""
    nt = U.shape[0]
    t0, t1 = slab_bounds(nt, world, rank)
    ts = [(t % nt) for t in range(t0 - 1, t1 + 1)]
    Ul = np.array(U[ts], copy=True)
    for i, t in enumerate(ts):
        if t == nt - 1 and bc[3] < 0:
            Ul[i, ..., 3, :, :] *= -1
    return Ul


def slab_vector(v, world, rank):
    """A global site-outer vector (numpy, (Nt, ...)) cut to the slab with its
    ghost slices (copies of the neighbours' edge slices)."""
    nt = v.shape[0]
    t0, t1 = slab_bounds(nt, world, rank)
    return np.ascontiguousarray(v[[(t % nt) for t in range(t0 - 1, t1 + 1)]])


class SlabOperator:
    """D on the owned slices of one slab (see the module docstring)."""

    def __init__(self, kind, U_global, nv, bc=(1, 1, 1, 1), prec=D.F32, world=1, rank=0,
                 layout=D.SITE_INNER, device=None):
        U_global = np.asarray(U_global)
        self.nt_global = U_global.shape[0]
        self.world, self.rank = world, rank
        self.t0, self.t1 = slab_bounds(self.nt_global, world, rank)
        self.nt_local = self.t1 - self.t0
        Ul = torch.from_numpy(slab_links(U_global, bc, world, rank))
        Ul = Ul.to(device) if device is not None else Ul.cuda()
        self.op = D.DiracOp(kind, Ul, nv, (bc[0], bc[1], bc[2], 1), prec, layout=layout)
        self.kind = kind
        nx, ny, nz, _ = self.op.dims
        self.slice_sites = nx * ny * nz
        self.wilson_type = kind in (D.WILSON, D.BRILLOUIN, D.WLAP, D.BLAP)
        self.half_spinor = kind == D.WILSON

    def projections(self, dagger):
        """(first, last): the projector signs the owned edge slices are packed
        with.  The D_W forward t-hop applies (1 - sgn gamma_4) to the slice
        above, the backward hop (1 + sgn gamma_4) to the slice below; a slab's
        first slice is its lower neighbour's upper ghost, its last slice the
        upper neighbour's lower ghost.  Full slices (0) for the other kinds."""
        if not self.half_spinor:
            return 0, 0
        sgn = -1 if dagger else 1
        return -sgn, sgn

    def pack(self, x, dagger=False):
        pf, pl = self.projections(dagger)
        lo = self.op.halo_pack(x, 1, self.op.halo_buffer(pf), pf)
        hi = self.op.halo_pack(x, self.nt_local, self.op.halo_buffer(pl), pl)
        return lo, hi

    def unpack(self, x, recv_lo, recv_hi, dagger=False):
        """recv_lo: the lower neighbour's last slice, recv_hi: the upper
        neighbour's first slice (as packed by `pack`)."""
        pf, pl = self.projections(dagger)
        self.op.halo_unpack(recv_lo, 0, x, pl)
        self.op.halo_unpack(recv_hi, self.nt_local + 1, x, pf)

    def apply_owned(self, x, out, m0, dagger=False):
        return self.op.apply_range(x, out, self.slice_sites, self.nt_local * self.slice_sites, m0=m0, dagger=dagger)

    def close(self):
        self.op.close()


def exchange(send_lo, send_hi, world, rank, group=None):
    """Send this slab's first slice to the lower neighbour and its last slice
    to the upper one (periodic ring); returns (from lower, from upper).  With
    NCCL the four transfers run as one batch (a pair of ranks posting sends
    before receives must not wait on each other); with gloo as tagged
    point-to-point messages.  world = 1 returns the slab's own slices."""
    if world == 1:
        return send_hi, send_lo
    import torch.distributed as dist
    prev, nxt = (rank - 1) % world, (rank + 1) % world
    recv_lo, recv_hi = torch.empty_like(send_hi), torch.empty_like(send_lo)
    if send_lo.is_cuda:
        # order per peer: the k-th send to a peer meets that peer's k-th receive
        # from us (world = 2 has prev == next): lo goes out first, hi second;
        # hi (from next) is received first, lo (from prev) second
        ops = [dist.P2POp(dist.isend, send_lo, prev, group), dist.P2POp(dist.isend, send_hi, nxt, group),
               dist.P2POp(dist.irecv, recv_hi, nxt, group), dist.P2POp(dist.irecv, recv_lo, prev, group)]
        for r in dist.batch_isend_irecv(ops):
            r.wait()
    else:
        reqs = [dist.isend(send_lo, prev, group, tag=0), dist.isend(send_hi, nxt, group, tag=1),
                dist.irecv(recv_hi, nxt, group, tag=0), dist.irecv(recv_lo, prev, group, tag=1)]
        for r in reqs:
            r.wait()
    return recv_lo, recv_hi


def apply_distributed(slab, x, out, m0, dagger=False, group=None):
    """One apply on a multi-process run (one slab per rank)."""
    lo, hi = slab.pack(x, dagger)
    torch.cuda.current_stream().synchronize()
    recv_lo, recv_hi = exchange(lo, hi, slab.world, slab.rank, group)
    slab.unpack(x, recv_lo, recv_hi, dagger)
    return slab.apply_owned(x, out, m0, dagger)


def apply_in_process(slabs, xs, outs, m0, dagger=False):
    """All slabs of one lattice held by one process (one GPU): pack every
    slab, hand each packed slice to its neighbour by a device copy, unpack,
    then apply on the owned slices.  No kernel waits on another; the host
    orders the steps."""
    R = len(slabs)
    packed = [s.pack(x, dagger) for s, x in zip(slabs, xs)]
    for r, (s, x) in enumerate(zip(slabs, xs)):
        s.unpack(x, packed[(r - 1) % R][1], packed[(r + 1) % R][0], dagger)
    for s, x, o in zip(slabs, xs, outs):
        s.apply_owned(x, o, m0, dagger)
    return outs


def _reduce_sum(parts, world, group):
    """Sum of per-slab partial reductions (device tensors of N_v entries):
    over the slabs held here, then over the ranks (all-reduce) when world > 1."""
    total = parts[0].clone()
    for t in parts[1:]:
        total += t
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(total, op=dist.ReduceOp.SUM, group=group)
    return total


def cg_normal(slabs, bs, m0, tol=1e-10, maxit=10000, group=None):
    """CG on the normal equations D^dag D x = D^dag b over a slab-decomposed
    lattice (Sec. 9's CG, one independent recurrence per RHS): every
    application of D and D^dag exchanges the halos, every dot product runs on
    the owned sites of each slab (dirac_vec_dot_range) and is summed over the
    slabs -- the all-reduce of N_v scalars per dot that a distributed solver
    adds.  `slabs`: every slab of the lattice held by this process (one GPU,
    the exchange a device copy), or this rank's single slab (one slab per
    rank, the exchange and the all-reduce over `group`).  bs: the slabs'
    right-hand sides (ghost slices are ignored).  Returns (xs, iterations,
    relative normal residual per RHS)."""
    import numpy as np
    R = len(slabs)
    nslab = slabs[0].world
    if R == nslab:
        distributed, world = False, 1        # every slab here: sums stay local
    elif R == 1:
        distributed, world = True, nslab     # one slab per rank: all-reduce
    else:
        raise ValueError("hold every slab of the lattice, or one slab per rank")
    nv = slabs[0].op.nv
    dev = slabs[0].op.device

    def owned(s):
        return s.slice_sites, s.nt_local * s.slice_sites

    def apply(xs, outs, dagger):
        if distributed:
            apply_distributed(slabs[0], xs[0], outs[0], m0, dagger, group)
        else:
            apply_in_process(slabs, xs, outs, m0, dagger)

    def norm2(vs):
        return _reduce_sum([s.op.norm2_range(v, *owned(s)) for s, v in zip(slabs, vs)], world, group)

    def dot_re(us, vs):
        return _reduce_sum([s.op.dot_range(u, v, *owned(s)).real.contiguous() for s, u, v in zip(slabs, us, vs)],
                           world, group)

    one = torch.ones(nv, dtype=torch.complex128, device=dev)
    zero = torch.zeros(nv, dtype=torch.complex128, device=dev)
    # the right-hand side D^dag b (b's halos are exchanged in a copy: b is not modified)
    bcopy = [s.op.axpby(one, b, zero, b) for s, b in zip(slabs, bs)]
    rhs = [s.op.new_vector() for s in slabs]
    apply(bcopy, rhs, True)
    xs = [s.op.new_vector() for s in slabs]
    rs = [s.op.axpby(one, h, zero, h) for s, h in zip(slabs, rhs)]
    ps = [s.op.axpby(one, h, zero, h) for s, h in zip(slabs, rhs)]
    ts = [s.op.new_vector() for s in slabs]
    aps = [s.op.new_vector() for s in slabs]
    nb = norm2(rhs).cpu().numpy()
    rr = nb.copy()
    done = nb == 0
    it = 0
    while it < maxit and not np.all(done | (np.sqrt(rr) < tol * np.sqrt(nb))):
        apply(ps, ts, False)
        apply(ts, aps, True)
        pap = dot_re(ps, aps).cpu().numpy()
        alpha = np.where(pap > 0, rr / np.where(pap > 0, pap, 1.0), 0.0)
        a = torch.from_numpy(alpha.astype(np.complex128)).to(dev)
        for s, x, p, r, ap in zip(slabs, xs, ps, rs, aps):
            s.op.axpby(one, x, a, p, x)          # x += alpha p
            s.op.axpby(one, r, -a, ap, r)        # r -= alpha A p
        rr_new = norm2(rs).cpu().numpy()
        beta = np.where(rr > 0, rr_new / np.where(rr > 0, rr, 1.0), 0.0)
        bt = torch.from_numpy(beta.astype(np.complex128)).to(dev)
        for s, p, r in zip(slabs, ps, rs):
            s.op.axpby(one, r, bt, p, p)         # p = r + beta p
        rr = rr_new
        it += 1
    relres = np.where(nb > 0, np.sqrt(rr / np.where(nb > 0, nb, 1.0)), 0.0)
    return xs, it, relres

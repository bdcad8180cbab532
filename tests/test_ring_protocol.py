"""CPU replay of the per-warp TMA rings of the streaming kernels: the order in
which a warp issues its boxes, waits for them, reads them and hands their
slots back, across the units (row runs of a column strip) it takes in turn.

Two disciplines are restated.
  - A ring that runs across units (k_stencil_rows, k_max_rows,
    k_interp_rows): kRing boxes issued up front, then one more each time a
    box is released; box q (in issue order) lives in slot q % kRing and
    completes phase q // kRing of that slot's mbarrier; the issue side walks
    the same units, in the same order, as the reading side.
  - A ring restarted per unit (k_harris_rows, k_chain_rows): the first kRing
    boxes of a unit issued when the unit starts, box j + kRing issued after
    box j has been read; box numbers continue across units (qbase).
For every wait the replay checks that the box waited for has been issued and
that nothing issued later has gone into its slot (a slot is refilled only
after it was read), so that the slot's mbarrier is in the phase the kernel's
parity names, and that the box holds the rows the reader expects.  Every box
issued is read exactly once, and no box is in flight when a warp ends.
Nothing here touches a GPU."""

import pytest


class Ring:
    """One warp's ring that runs across units: issue side and slot state."""

    def __init__(self, kring, units, nbox, stride, gw):
        self.kring, self.units, self.nbox, self.stride = kring, units, nbox, stride
        self.issued = self.released = 0
        self.iu, self.ij = gw, 0
        self.slot = {}            # slot -> (box number, unit, box within unit)
        self.log = []

    def issue(self):
        if self.iu >= self.units:
            return
        q = self.issued
        s = q % self.kring
        if s in self.slot:        # the slot's previous box has been handed back
            assert self.slot[s][0] < self.released, ("slot refilled before it was read", s, q)
        self.slot[s] = (q, self.iu, self.ij)
        self.log.append((self.iu, self.ij))
        self.issued += 1
        self.ij += 1
        if self.ij == self.nbox(self.iu):
            self.ij = 0
            self.iu += self.stride


def replay_running_ring(kring, units, nbox, stride, gw, reads_of):
    """reads_of(u): the boxes unit u reads, in order (box within the unit)."""
    R = Ring(kring, units, nbox, stride, gw)
    for _ in range(kring):
        R.issue()
    consumed = []
    for u in range(gw, units, stride):
        q = R.released
        for j in reads_of(u):
            assert q < R.issued, ("waited for a box never issued", u, j)
            box, bu, bj = R.slot[q % kring]
            assert box == q, ("the slot holds another box", q, box)
            assert (bu, bj) == (u, j), ("box holds other rows", (bu, bj), (u, j))
            consumed.append((u, j))
            q += 1
            R.released = q
            R.issue()
    assert R.issued == R.released, "boxes still in flight when the warp ends"
    assert consumed == R.log
    return len(consumed)


def stencil_rows_case(H, rows, strips, planes):
    runs = -(-H // rows)
    units = strips * runs * planes

    def n_in(u):
        oy = ((u % (strips * runs)) // strips) * rows
        return min(rows, H - oy) + 4

    return units, (lambda u: -(-n_in(u) // 4)), (lambda u: range(-(-n_in(u) // 4)))


def max_rows_case(H, rows, strips, planes, ry):
    runs = -(-H // rows)
    units = strips * runs * planes

    def n_in(u):
        y0 = ((u % (strips * runs)) // strips) * rows
        return min(rows, H - y0) + 2 * ry

    return units, (lambda u: -(-n_in(u) // 4)), (lambda u: range(-(-n_in(u) // 4)))


def interp_case(CH, rows, strips):
    runs = -(-CH // rows)
    units = strips * runs

    def inrun(u):
        return min(rows, CH - (u // strips) * rows)

    return units, inrun, (lambda u: range(inrun(u)))


@pytest.mark.parametrize("H,rows,strips,planes", [(1, 1, 1, 1), (5, 3, 2, 3), (37, 8, 3, 1), (1536, 20, 22, 3),
                                                  (100, 100, 5, 2), (7, 64, 4, 3)])
@pytest.mark.parametrize("warps,blocks", [(1, 1), (4, 3), (8, 19)])
def test_running_rings(H, rows, strips, planes, warps, blocks):
    stride = warps * blocks
    cases = [("stencil", 3, stencil_rows_case(H, rows, strips, planes))]
    cases += [("max r%d" % ry, 3, max_rows_case(H, rows, strips, planes, ry)) for ry in (0, 1, 4)]
    cases += [("interp", 3, interp_case(H, rows, strips))]
    for name, kring, (units, nbox, reads_of) in cases:
        total = 0
        for gw in range(min(stride, units)):
            total += replay_running_ring(kring, units, nbox, stride, gw, reads_of)
        assert total == sum(nbox(u) for u in range(units)), name


def replay_unit_ring(kring, unit_list, geom_of, box_rows):
    """Per-unit ring: returns the boxes read, checking every wait.
    geom_of(u) = (steps, input rows inside the image)."""
    slot = {}
    qbase = 0
    read = []
    for u in unit_list:
        n, n_in = geom_of(u)
        nbox = -(-n_in // box_rows)
        issued = set()

        def issue(j):
            q = qbase + j
            s = q % kring
            if s in slot:
                assert slot[s][1], ("slot refilled before it was read", s, q)
            slot[s] = [q, False, (u, j)]
            issued.add(j)

        for j in range(min(kring, nbox)):
            issue(j)
        j = 0
        while box_rows * j < n:
            if box_rows * j < n_in:                 # the kernel's test: a box to wait for
                assert j < nbox
                q = qbase + j
                assert j in issued, ("waited for a box never issued", u, j)
                box, was_read, ident = slot[q % kring]
                assert box == q and not was_read and ident == (u, j)
                slot[q % kring][1] = True
                read.append((u, j))
            if j + kring < nbox:
                issue(j + kring)
            j += 1
        assert issued == set(range(nbox)), ("boxes of the unit never issued", u)
        assert all(v[1] for v in slot.values()), "a box in flight at the end of a unit"
        qbase += nbox
    return read


@pytest.mark.parametrize("H,rows", [(1, 1), (2, 5), (9, 4), (37, 14), (1536, 20), (130, 129)])
@pytest.mark.parametrize("stride,gw", [(1, 0), (5, 2), (38, 37)])
def test_per_unit_rings(H, rows, stride, gw):
    strips = 3
    runs = -(-H // rows)
    units = list(range(gw, strips * runs, stride))

    # k_harris_rows: boxes of 2 rows; rows read from y0 = max(oy - 2, 0), steps
    # to ye + 2, rows inside the image only
    def harris(u):
        oy = (u // strips) * rows
        ye, y0 = min(oy + rows, H), max(oy - 2, 0)
        n_steps = ye - y0 + 2
        n_in = min(y0 + n_steps, H) - y0
        return n_steps, n_in

    got = replay_unit_ring(4, units, harris, 2)
    assert len(got) == sum(-(-harris(u)[1] // 2) for u in units)

    # k_chain_rows: boxes of 4 rows, halo 2D rows
    for D in (2, 4):
        def chain(u, D=D):
            oy = (u // strips) * rows
            ye, y0 = min(oy + rows, H), max(oy - 2 * D, 0)
            n_steps = ye - y0 + 2 * D
            n_in = min(y0 + n_steps, H) - y0
            return n_steps, n_in

        got = replay_unit_ring(3, units, chain, 4)
        assert len(got) == sum(-(-chain(u)[1] // 4) for u in units)


def test_running_ring_catches_an_overfull_ring():
    # a mistake planted in the restated discipline (one box more issued up
    # front than the ring has slots) must fail the replay
    units, nbox, reads_of = stencil_rows_case(37, 8, 3, 1)
    R = Ring(3, units, nbox, 1, 0)
    with pytest.raises(AssertionError):
        for _ in range(4):
            R.issue()

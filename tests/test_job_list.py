"""The mixed deposit's hand-out of grid points to lanes, checked on the CPU: a model of
one warp and block of the kernel's enumeration (each lane owns PIX pixel slots; a slot's
run is the grid points its pixel reaches in the block; an inclusive prefix sum over the
warp gives every slot its job offset; the first kJobTable jobs are listed as (slot, grid
point) by their owners; job t beyond the table finds its slot as the last one whose
offset is <= t, by bisection over the lane-major slot offsets; runs above the warp limit
stay with their owners) yields every (slot, grid point) of every run exactly once."""
import numpy as np
import pytest

LANES = 32
PIX = 2            # pixels per thread of the mixed deposit
TABLE = 128        # jobs listed explicitly per warp and block


def _jobs(runs, first, max_warp):
    """(slot, grid point) of every job, in the order the warp's lanes take them."""
    n_slots = LANES * PIX
    K = [[k if k <= max_warp else 0 for k in row] for row in runs]
    big = [[k if k > max_warp else 0 for k in row] for row in runs]
    tot = [sum(row) for row in K]
    incl = list(np.cumsum(tot))
    T = int(incl[-1])
    s_kp, s_ja, s_tab = [0] * n_slots, [0] * n_slots, [None] * TABLE
    for lane in range(LANES):
        run = int(incl[lane]) - tot[lane]
        for q in range(PIX):
            sl = lane * PIX + q
            s_kp[sl] = run
            s_ja[sl] = first[lane][q]
            for t in range(K[lane][q]):
                if run + t < TABLE:
                    s_tab[run + t] = (sl, first[lane][q] + t)
            run += K[lane][q]

    def slot_of(t):
        pos, step = 0, 16 * PIX
        while step > 0:
            if s_kp[pos + step] <= t:
                pos += step
            step >>= 1
        return pos

    out = []
    for lane in range(LANES):
        for t in range(lane, T, LANES):
            if t < TABLE:
                out.append(s_tab[t])
            else:
                sl = slot_of(t)
                out.append((sl, s_ja[sl] + (t - s_kp[sl])))
    for lane in range(LANES):
        for q in range(PIX):
            out.extend((lane * PIX + q, first[lane][q] + t) for t in range(big[lane][q]))
    return out


def _cases():
    rng = np.random.Generator(np.random.PCG64(20220607))
    zeros = np.zeros((LANES, PIX), int)
    one = zeros.copy()
    one[17, 1] = 700                       # one pixel reaches everything, past the table
    last = zeros.copy()
    last[31, 1] = 5                        # only the warp's last slot has work
    first = zeros.copy()
    first[0, 0] = 3
    edge = np.full((LANES, PIX), 2)        # exactly the table: 64 slots x 2
    yield "empty", zeros
    yield "single_slot", one
    yield "last_slot", last
    yield "first_slot", first
    yield "table_edge", edge
    yield "table_edge_plus_one", edge + (np.arange(LANES * PIX).reshape(LANES, PIX) == 40)
    for i in range(6):                     # about 1 grid point per pixel and block
        yield f"poisson_{i}", rng.poisson(1.1, (LANES, PIX))
    for i in range(4):                     # sparse long runs with zero slots between
        yield f"sparse_{i}", rng.poisson(9.0, (LANES, PIX)) * (rng.random((LANES, PIX)) < 0.2)
    yield "over_warp_limit", np.where(rng.random((LANES, PIX)) < 0.1, 60, 1)


@pytest.mark.parametrize("name,runs", list(_cases()))
def test_every_grid_point_of_every_run_is_taken_once(name, runs):
    rng = np.random.Generator(np.random.PCG64(len(name)))
    first = rng.integers(0, 65536, (LANES, PIX)).tolist()
    got = _jobs(runs.tolist(), first, max_warp=50)
    want = [(lane * PIX + q, first[lane][q] + t)
            for lane in range(LANES) for q in range(PIX) for t in range(int(runs[lane, q]))]
    assert sorted(got) == sorted(want)


def test_offsets_are_monotone_in_slot_order():
    """The bisection needs the job offsets non-decreasing over the warp's slots: the
    owner writes a lane's PIX offsets in pixel order after the exclusive prefix of the
    lanes before it."""
    rng = np.random.Generator(np.random.PCG64(7))
    runs = rng.poisson(2.0, (LANES, PIX))
    tot = runs.sum(1)
    excl = np.concatenate([[0], np.cumsum(tot)[:-1]])
    offsets = (excl[:, None] + np.concatenate([np.zeros((LANES, 1), int),
                                               np.cumsum(runs, 1)[:, :-1]], 1)).ravel()
    assert (np.diff(offsets) >= 0).all()

"""Host check of the AA scheme's index algebra (no GPU): on a small D3Q19 lattice with walled
and periodic faces, a plain numpy model of the two AA steps and of the pair-swap
normalisation reproduces ping-pong streaming with halfway bounce-back, step after step, and
each site of either AA step writes exactly the locations it reads, no location being touched
by two sites.  The collision is a fixed random linear map per site (the layout question does
not depend on what the collision computes).  The model follows the layouts described for the
scheme: swapped (plane opp(i) at x holds f*_i(x)) and streamed (plane i at x holds the f_i(x)
a pull gathers there, or the raw f*_opp(i)(x) where that pull crosses a wall)."""
import itertools

import numpy as np
import pytest


def _lattice(orc, shape, periodic):
    e = np.asarray(orc.tables()["e19"]).T.astype(int)  # (19, 3): velocities of Eq. 19
    opp = [int(np.flatnonzero((e == -e[i]).all(axis=1))[0]) for i in range(19)]
    nx, ny, nz = shape
    sites = list(itertools.product(range(nx), range(ny), range(nz)))
    index = {s: k for k, s in enumerate(sites)}

    def source(x, i):
        """x - e_i with periodic wrap, or None across a wall."""
        out = []
        for a in range(3):
            c = x[a] - e[i][a]
            if c < 0 or c >= shape[a]:
                if not periodic[a]:
                    return None
                c %= shape[a]
            out.append(c)
        return tuple(out)

    return e, opp, sites, index, source


def _pingpong_step(fstar, A, sites, index, source, opp):
    f = np.empty_like(fstar)
    for x in sites:
        k = index[x]
        for i in range(19):
            src = source(x, i)
            f[i, k] = fstar[opp[i], k] if src is None else fstar[i, index[src]]
    # the collision per site, as the AA model applies it (the same sums in the same order)
    return np.stack([A @ f[:, k] for k in range(f.shape[1])], axis=1)


def _aa_pull(P, A, sites, index, source, opp, log):
    """Swapped -> streamed.  Reads P[opp(i), x - e_i] (or P[i, x] across a wall), pushes
    f*_j to P[j, x + e_j] (or P[opp(j), x])."""
    gathered, reads = {}, {}
    for x in sites:
        k = index[x]
        f = np.empty(19)
        rs = set()
        for i in range(19):
            src = source(x, i)
            loc = (i, k) if src is None else (opp[i], index[src])
            f[i] = P[loc]
            rs.add(loc)
        gathered[x] = A @ f
        reads[x] = rs
    for x in sites:  # every read happens before any write, as in one kernel launch
        k = index[x]
        ws = set()
        for j in range(19):
            dst = source(x, opp[j])  # x + e_j
            loc = (opp[j], k) if dst is None else (j, index[dst])
            P[loc] = gathered[x][j]
            ws.add(loc)
        log.append((reads[x], ws))


def _aa_local(P, A, sites, index, opp, log):
    """Streamed -> swapped.  Own-site planes only (halfway bounce-back needs no rule on the raw
    value: the pulled population across a wall is f*_opp(i)(x) itself)."""
    for x in sites:
        k = index[x]
        fstar = A @ P[:, k]
        P[:, k] = fstar[opp]
        log.append(({(i, k) for i in range(19)}, {(i, k) for i in range(19)}))


def _normalise(P, sites, index, source, opp):
    """Streamed -> swapped by swapping each pair (P[j, x + e_j], P[opp(j), x]) once."""
    for x in sites:
        k = index[x]
        for j in range(19):
            if j < opp[j]:
                dst = source(x, opp[j])
                if dst is not None:
                    a, b = (j, index[dst]), (opp[j], k)
                    P[a], P[b] = P[b], P[a]


def _check_disjoint(log):
    owner = {}
    for site_no, (reads, writes) in enumerate(log):
        assert reads == writes  # a site writes exactly what it reads
        for loc in writes:
            assert owner.setdefault(loc, site_no) == site_no  # no location shared by two sites


@pytest.mark.parametrize("shape,periodic", [((4, 3, 2), (False, True, False)),
                                            ((3, 1, 5), (True, False, True)),
                                            ((2, 4, 1), (False, False, True))])
def test_aa_steps_reproduce_pingpong(orc, shape, periodic):
    e, opp, sites, index, source = _lattice(orc, shape, periodic)
    rng = np.random.default_rng(7)
    A = np.eye(19) + 0.1 * rng.standard_normal((19, 19))
    fstar = rng.standard_normal((19, len(sites)))  # post-collision state, ping-pong layout
    P = fstar[opp, :].copy()                        # the same state, swapped layout
    for step in range(6):
        fstar = _pingpong_step(fstar, A, sites, index, source, opp)
        log = []
        if step % 2 == 0:
            _aa_pull(P, A, sites, index, source, opp, log)
            # read the state as a reader would: rearranged into the swapped layout
            Q = P.copy()
            _normalise(Q, sites, index, source, opp)
            assert np.array_equal(Q[opp, :], fstar)
        else:
            _aa_local(P, A, sites, index, opp, log)
            assert np.array_equal(P[opp, :], fstar)
        _check_disjoint(log)

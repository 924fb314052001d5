"""The column ordering of the register kernels for more columns than lanes
(k_eig_wide, k_qstep_wide): lane i < N/2 holds a column pair (top_i, bot_i);
between rounds every column but top_0 moves one step along the ring
top_1 .. top_{H-1}, bot_{H-1} .. bot_0, the way ring_step moves them with one
shuffle up and one shuffle down per row (lane 0 sends its bottom column up,
lane H-1 keeps its top column as its new bottom one).  A sweep of the
one-sided Jacobi method must rotate every pair of columns once and leave every
column where it started (the kernels read the final columns by position).
The emulation follows the lane-level moves, including what the idle lanes
>= H hold, for every column count the kernels are instantiated with."""
import pytest

LANES = 32


def ring_step(top, bot, H):
    """One move of all 32 lanes, as the kernels' shuffles do it."""
    send_up = [bot[l] if l == 0 else top[l] for l in range(LANES)]
    up = [send_up[l - 1] if l >= 1 else send_up[l] for l in range(LANES)]  # __shfl_up_sync(.., 1)
    dn = [bot[l + 1] if l + 1 < LANES else bot[l] for l in range(LANES)]  # __shfl_down_sync(.., 1)
    new_top = [top[l] if l == 0 else up[l] for l in range(LANES)]
    new_bot = [top[l] if l == H - 1 else dn[l] for l in range(LANES)]
    return new_top, new_bot


@pytest.mark.parametrize("N", [34, 40, 48, 50, 56, 60, 64])
def test_every_pair_meets_once_per_sweep_and_columns_return(N):
    H = N // 2
    top = list(range(H)) + [None] * (LANES - H)
    bot = [H + i for i in range(H)] + [None] * (LANES - H)
    seen = {}
    for rnd in range(N - 1):
        for lane in range(H):
            a, b = top[lane], bot[lane]
            assert a is not None and b is not None
            key = frozenset((a, b))
            assert len(key) == 2
            assert key not in seen, (N, rnd, lane, a, b, seen.get(key))
            seen[key] = rnd
        top, bot = ring_step(top, bot, H)
    assert len(seen) == N * (N - 1) // 2
    assert top[:H] == list(range(H))
    assert bot[:H] == [H + i for i in range(H)]


def test_moves_never_read_from_idle_lanes():
    # an active lane's new columns come from lanes < H only (idle lanes may
    # hold copies, never originals the active lanes need)
    for N in (34, 40, 64):
        H = N // 2
        top = [("t", l) if l < H else ("idle", l) for l in range(LANES)]
        bot = [("b", l) if l < H else ("idle", l) for l in range(LANES)]
        for _ in range(2 * N):
            top, bot = ring_step(top, bot, H)
            assert all(top[l][0] != "idle" and bot[l][0] != "idle" for l in range(H))

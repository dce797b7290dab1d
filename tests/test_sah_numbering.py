"""The numbering the SAH-top builder gives its top nodes (no GPU): in any
binary tree over an ordered sequence of n leaves, numbering every left child
by the position of its last leaf, every right child by the position of its
first leaf and the root 0 gives the n - 1 inner nodes the numbers 0 .. n - 2,
each once.  The builder relies on it to number nodes without a counter; here
it is checked on random trees of every shape the splits can make (balanced,
chains, random cuts), so that a wrong side or an off-by-one fails."""
import random

import pytest


def _numbers(n, cut):
    """Inner-node numbers of the tree that `cut(b, e)` splits range [b, e)
    into [b, m) and [m, e), recursively down to single leaves."""
    out = []
    stack = [(0, n, 0)]  # range, number given by its parent
    while stack:
        b, e, num = stack.pop()
        if e - b < 2:
            continue
        out.append(num)
        m = cut(b, e)
        assert b < m < e
        stack.append((b, m, m - 1))  # left child: its last position
        stack.append((m, e, m))      # right child: its first position
    return out


@pytest.mark.parametrize("shape", ["middle", "left_chain", "right_chain", "random"])
def test_top_node_numbers_are_a_bijection(shape):
    rng = random.Random(7)
    for n in list(range(2, 70)) + [rng.randint(70, 5000) for _ in range(40)]:
        cut = {"middle": lambda b, e: b + (e - b) // 2,
               "left_chain": lambda b, e: e - 1,
               "right_chain": lambda b, e: b + 1,
               "random": lambda b, e: rng.randint(b + 1, e - 1)}[shape]
        nums = _numbers(n, cut)
        assert sorted(nums) == list(range(n - 1)), (shape, n)

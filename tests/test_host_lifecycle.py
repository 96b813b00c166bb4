"""Host logic of the lifecycle: identities carried through the densify /
prune rows, and the training labels built from the plain criterion's later
chunks (a Gaussian pruned in this or any later chunk is a prune example, only
Gaussians the chunk saw carry labels)."""
import numpy as np
import torch

from paper_2606_30436_b300.lifecycle import carry_ids, future_labels


def test_carry_ids_follows_the_rows():
    ids = np.array([10, 11, 12, 13, 14])
    dens = np.array([0, 1, 0, 1, 0], np.uint8)
    prune = np.array([0, 0, 1, 1, 0], np.uint8)  # 13 is both: pruning wins, it emits nothing
    out, nxt = carry_ids(ids, dens, prune, 100)
    assert out.tolist() == [10, 11, 100, 14] and nxt == 101
    out2, nxt2 = carry_ids(out, np.array([1, 0, 1, 0], np.uint8), np.zeros(4, np.uint8), nxt)
    assert out2.tolist() == [10, 101, 11, 100, 102, 14] and nxt2 == 103
    empty, n3 = carry_ids(np.array([], np.int64), np.array([], np.uint8), np.array([], np.uint8), 7)
    assert len(empty) == 0 and n3 == 7


def _u8(a):
    return torch.tensor(a, dtype=torch.uint8)


def test_future_prune_labels():
    feat = torch.zeros(16, 4)
    # chunk 0: ids 0..3, nothing pruned, 3 unseen; chunk 1: ids 0, 1, 3, 5, prunes 1; chunk 2: ids 0, 3, 5, prunes 3
    s0 = (feat, 4, _u8([1, 0, 0, 0]), _u8([0, 0, 0, 0]), torch.tensor([True, True, True, False]), np.array([0, 1, 2, 3]))
    s1 = (feat, 4, _u8([0, 0, 0, 0]), _u8([0, 1, 0, 0]), torch.tensor([True, True, True, True]), np.array([0, 1, 3, 5]))
    s2 = (feat, 3, _u8([0, 0, 1]), _u8([0, 1, 0]), torch.tensor([True, True, False]), np.array([0, 3, 5]))
    rows = future_labels([s0, s1, s2], device="cpu")
    assert [r[1] for r in rows] == [4, 4, 3]
    # chunk 0: 1 pruned at chunk 1 -> label; 3 pruned at chunk 2 but unseen in chunk 0 -> no label
    assert rows[0][3].tolist() == [0, 1, 0, 0] and rows[0][2].tolist() == [1, 0, 0, 0]
    assert rows[1][3].tolist() == [0, 1, 1, 0]
    assert rows[2][3].tolist() == [0, 1, 0] and rows[2][2].tolist() == [0, 0, 0]  # id 5's densify bit: unseen

"""Oracle of the recursive re-labeling at tissue boundaries (Sec. 2.1.3 item 2,
Fig. 3).

TEST INFRASTRUCTURE ONLY (see the package docstring).

After the nodes of a labeled mesh have changed (moved, or the surfaces were
replaced), the labels are repaired at the tissue boundaries instead of
re-labeling every node.  One pass, in the paper's order:
  1. the tissue boundary is the set of tets whose four node labels are not
     all equal;
  2. the solid angle is re-evaluated for the nodes of those tets;
  3. the node labels are updated, which can move the boundary;
repeated until a pass changes no node label (the boundary no longer changes,
Fig. 3) or the pass limit is reached.

Reading where the paper is silent: a node is re-evaluated at most once per
call (its position is fixed during the call, so a second evaluation would
return the same label); a pass with no node left to evaluate changes nothing
and ends the recursion.
"""
from __future__ import annotations

import numpy as np

from . import label_points


def relabel_boundary(nodes, tets, labels, surfaces, priority, max_passes: int):
    """Returns (labels, per_pass [(evaluated, changed), ...], converged)."""
    nodes = np.asarray(nodes, dtype=np.float32).reshape(-1, 3)
    tets = np.asarray(tets, dtype=np.int64).reshape(-1, 4)
    labels = np.array(labels, dtype=np.int32, copy=True)
    if tets.size and (tets.min() < 0 or tets.max() >= nodes.shape[0]):
        raise ValueError("tet node index out of range")
    fresh = np.zeros(nodes.shape[0], dtype=bool)
    per_pass = []
    converged = False
    for _ in range(max_passes):
        lt = labels[tets]
        boundary = (lt != lt[:, :1]).any(axis=1)
        cand = np.unique(tets[boundary].ravel())
        cand = cand[~fresh[cand]]
        changed = 0
        if cand.size:
            new, _ = label_points(nodes[cand], surfaces, priority)
            fresh[cand] = True
            changed = int((new != labels[cand]).sum())
            labels[cand] = new
        per_pass.append((int(cand.size), changed))
        if changed == 0:
            converged = True
            break
    return labels, per_pass, converged

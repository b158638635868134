"""Test-side chains for the two-level (node grid a x GPU grid b) mappings.

Written for the tests from the mapping's definition, independently of the
engine's own chain builder: node u_t = floor(x_t a_t / L_t); GPU coordinate
floor(x_t a_t b_t / L_t) mod b_t (block within the node, Fig. 5b) or
x_t mod b_t (cyclic within the node, Appendix A.1).
"""


def hier_chain(k, a, b, variant):
    """Split/swap/merge chain on Machine(n, g) whose final space realises the
    two-level mapping: node dimension split by a, GPU dimension by b; for
    the block variant each pair (b_t, a_t) is merged (GPU digit fastest) so
    that a block distribution over the product grid gives node w_t div b_t,
    GPU w_t mod b_t; for the cyclic variant the 2k-D space is the
    hierarchical distribution's (Appendix A.1)."""
    ch = [("split", i, a[i]) for i in range(k - 1)]
    ch += [("split", k + j, b[j]) for j in range(k - 1)]
    if variant == "cyclic":
        return ch, ("hier",)
    labels = [("u", t) for t in range(k)] + [("v", t) for t in range(k)]
    want = [lab for t in range(k) for lab in (("v", t), ("u", t))]
    for pos in range(2 * k):
        j = labels.index(want[pos])
        if j != pos:
            ch.append(("swap", pos, j))
            labels[pos], labels[j] = labels[j], labels[pos]
    ch += [("merge", t, t + 1) for t in range(k)]
    return ch, ("block",)


def node_chain(k, a):
    ch = [("split", i, a[i]) for i in range(k - 1)]
    return ch + [("merge", k - 1, k)]

"""Text fixtures with values the paper prints (task graphs of Fig. 3 and Fig. 4)."""
import os

HERE = os.path.dirname(os.path.abspath(__file__))


def _task(tok):
    return (tok[0], int(tok[1]), int(tok[2]), int(tok[3]))


def read_graph_fixture(name):
    nodes, edges, tagged = [], [], []
    with open(os.path.join(HERE, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            tok = line.split()
            if tok[0] == "node":
                nodes.append(_task(tok[1:5]))
            else:
                a = _task(tok[1:5])
                assert tok[5] == "->"
                b = _task(tok[6:10])
                if tok[0] == "edge":
                    edges.append((a, b))
                else:
                    tagged.append((tok[0], a, b))
    return nodes, edges, tagged

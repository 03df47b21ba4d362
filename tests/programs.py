"""Datalog programs used by the tests and the benchmark, as plain data.

A rule is (head, body, variable_order); an atom is (relation, [terms]); a term is a
str (variable) or an int (constant).  The oracle ignores the variable order."""

TC = [
    (("Reach", ["x", "y"]), [("E", ["x", "y"])], ["x", "y"]),
    (("Reach", ["x", "z"]), [("Reach", ["x", "y"]), ("E", ["y", "z"])], ["x", "y", "z"]),
]
TC_RELS = {"E": 2, "Reach": 2}

TRI = [
    (("Tri", ["x", "y", "z"]), [("E", ["x", "y"]), ("E", ["y", "z"]), ("E", ["x", "z"])], ["x", "y", "z"]),
]
TRI_RELS = {"E": 2, "Tri": 3}

Q4 = [
    (("Q4", ["w", "x", "y", "z"]),
     [("E", ["w", "x"]), ("E", ["w", "y"]), ("E", ["w", "z"]),
      ("E", ["x", "y"]), ("E", ["x", "z"]), ("E", ["y", "z"])],
     ["w", "x", "y", "z"]),
]
Q4_RELS = {"E": 2, "Q4": 4}

# Reach + Tri over one edge relation (the small plain-method workload).
TC_TRI = TC + TRI
TC_TRI_RELS = {"E": 2, "Reach": 2, "Tri": 3}

# Andersen-style points-to (Load is (v, w, f), Store is (v, f, w)).
POINTS_TO = [
    (("VPT", ["v", "h"]), [("New", ["v", "h"])], ["v", "h"]),
    (("VPT", ["v", "h"]), [("Assign", ["v", "w"]), ("VPT", ["w", "h"])], ["w", "v", "h"]),
    (("FPT", ["h1", "f", "h2"]),
     [("Store", ["v1", "f", "v2"]), ("VPT", ["v1", "h1"]), ("VPT", ["v2", "h2"])],
     ["v1", "h1", "f", "v2", "h2"]),
    (("VPT", ["v", "h2"]),
     [("Load", ["v", "w", "f"]), ("VPT", ["w", "h1"]), ("FPT", ["h1", "f", "h2"])],
     ["w", "h1", "f", "v", "h2"]),
]
POINTS_TO_RELS = {"New": 2, "Assign": 2, "Load": 3, "Store": 3, "VPT": 2, "FPT": 3}

# Same Generation (the paper's Table 3 workload): x and y are siblings, or children of a
# same-generation pair.
SG = [
    (("SG", ["x", "y"]), [("Edge", ["p", "x"]), ("Edge", ["p", "y"])], ["p", "x", "y"]),
    (("SG", ["x", "y"]), [("Edge", ["a", "x"]), ("SG", ["a", "b"]), ("Edge", ["b", "y"])], ["a", "b", "x", "y"]),
]
SG_RELS = {"Edge": 2, "SG": 2}

# Virtual-call resolution of a Java points-to analysis (the paper's CallGraphEdge example,
# Section 5): six atoms, eight variables; HeapAllocationType and MethodLookup (positions 4
# and 5) are the atoms the paper factors into a helper relation.
CGE = [
    (("CallGraphEdge", ["i", "m"]),
     [("Reachable", ["j"]), ("InstructionMethod", ["i", "j"]), ("VirtualMethodInvoc", ["i", "b", "sn", "dsc"]),
      ("VarPointsTo", ["h", "b"]), ("HeapAllocationType", ["h", "t"]), ("MethodLookup", ["sn", "dsc", "t", "m"])],
     ["j", "i", "b", "sn", "dsc", "h", "t", "m"]),
]
CGE_RELS = {"Reachable": 1, "InstructionMethod": 2, "VirtualMethodInvoc": 4, "VarPointsTo": 2,
            "HeapAllocationType": 2, "MethodLookup": 4, "CallGraphEdge": 2}
CGE_SPLIT = (4, 5)
# the same split written out by hand: helper over the variables shared with the rest
CGE_HELPER = [
    (("HelpNT", ["sn", "dsc", "h", "m"]),
     [("HeapAllocationType", ["h", "t"]), ("MethodLookup", ["sn", "dsc", "t", "m"])],
     ["sn", "dsc", "h", "t", "m"]),
    (("CallGraphEdge", ["i", "m"]),
     [("Reachable", ["j"]), ("InstructionMethod", ["i", "j"]), ("VirtualMethodInvoc", ["i", "b", "sn", "dsc"]),
      ("VarPointsTo", ["h", "b"]), ("HelpNT", ["sn", "dsc", "h", "m"])],
     ["j", "i", "b", "sn", "dsc", "h", "m"]),
]

# Comparisons and stratified negation (the extension Table 1 lists; semantics fixed by the
# oracle's reading).  Oriented cliques count each clique once.
TRI_LT = [(("TriLt", ["x", "y", "z"]),
           [("E", ["x", "y"]), ("E", ["y", "z"]), ("E", ["x", "z"]), ("<", "x", "y"), ("<", "y", "z")],
           ["x", "y", "z"])]
Q4_LT = [(("Q4Lt", ["w", "x", "y", "z"]),
          [("E", ["w", "x"]), ("E", ["w", "y"]), ("E", ["w", "z"]), ("E", ["x", "y"]), ("E", ["x", "z"]),
           ("E", ["y", "z"]), ("<", "w", "x"), ("<", "x", "y"), ("<", "y", "z")],
          ["w", "x", "y", "z"])]
# vertices, their reachability, and the pairs that do not reach each other
UNREACH = TC + [
    (("Node", ["x"]), [("E", ["x", "y"])], ["x", "y"]),
    (("Node", ["y"]), [("E", ["x", "y"])], ["x", "y"]),
    (("Unreach", ["x", "y"]), [("Node", ["x"]), ("Node", ["y"]), ("not", ("Reach", ["x", "y"]))], ["x", "y"]),
]
UNREACH_RELS = {"E": 2, "Reach": 2, "Node": 1, "Unreach": 2}

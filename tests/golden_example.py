"""Reader for the worked example of Table 1 (tests/golden/table1_worked_example.txt)."""
import os

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table1_worked_example.txt")


def load():
    sections, cur = {}, None
    with open(PATH) as f:
        for line in f:
            line = line.rstrip("\n")
            if not line or line.startswith("#"):
                continue
            if line.startswith("["):
                cur = line.strip("[]")
                sections[cur] = []
            else:
                sections[cur].append(line.split(" "))
    return sections


class Dictionary:
    """Test-side term dictionary: strings <-> uint32 ids."""

    def __init__(self):
        self.ids, self.terms = {}, []

    def id(self, term):
        if term not in self.ids:
            self.ids[term] = len(self.terms)
            self.terms.append(term)
        return self.ids[term]

    def term(self, i):
        return self.terms[int(i)]

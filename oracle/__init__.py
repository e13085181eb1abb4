"""CPU oracle for the word RASP (test infrastructure; see oracle.py)."""
